/*
 * plss.h -- C ABI of the GB300 (sm_103a) PLSS library, libplss.so.
 *
 * PLSS (Brust & Saunders, "PLSS: a projected linear systems solver",
 * arXiv 2207.07615) solves consistent systems A x = b, b in range(A), with A
 * sparse and m x n of any shape (Sec. 1, eq:axb). Two sketches are offered:
 *   - residual sketch S_k = [r_0 ... r_{k-1}] (Sec. 4, eq:S): the 1-step
 *     recursion of Theorem 4.1 as laid out in Algorithm 1 (Sec. 5), with an
 *     optional diagonal weight W (Sec. 4.1, eq:pkShortW);
 *   - identity sketch S_k = [e_{i_1} ... e_{i_k}] (Sec. 7, eq:pkKacz), the
 *     generalised Kaczmarz method, with a history window of K updates;
 *   - general sketch S_k = [s_1 ... s_k] (Sec. 2, eq:genS) of random sign
 *     columns, with the update of Corollary 2.2 (Sec. 2.4) and a history
 *     of at most K directions.
 *
 * Conventions for every entry point:
 *   - Nothing is thrown across the ABI; each call returns a plss_status and
 *     plss_last_error() gives a message for the calling thread.
 *   - The caller owns every pointer it passes and may free it once the call
 *     returns; the library copies what it keeps. The library owns the device
 *     memory it allocates for a context and frees it in plss_destroy.
 *   - Host/device: arrays are host memory unless the flag next to them
 *     (plss_csr.on_device, plss_opts.io_device) says device memory of the
 *     current CUDA device.
 *   - Indexing is 0-based. row_ptr is int64 with row_ptr[0] = 0,
 *     row_ptr[m] = nnz, non-decreasing; col_idx are int32 in [0, n), strictly
 *     increasing within each row. A context holds at most 2^31 - 1 nonzeros
 *     and rows/columns in total (larger inputs return PLSS_ERR_INVALID).
 *   - Distinct contexts may be used from different host threads; one
 *     context must not be used by two threads at once.
 */
#ifndef PLSS_H
#define PLSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLSS_OK = 0,              /* converged: ||r||/||b|| <= tol              */
    PLSS_NOT_CONVERGED = 1,   /* maxit reached; x is the last iterate      */
    PLSS_PENDING = 2,         /* plss_poll: request not finished yet        */
    PLSS_ERR_INVALID = -1,    /* bad argument or malformed CSR              */
    PLSS_ERR_NOMEM = -2,      /* device or host allocation failed           */
    PLSS_ERR_CUDA = -3,       /* a CUDA runtime call failed                 */
    PLSS_ERR_BREAKDOWN = -4,  /* recursion broke down (see plss_solve)      */
    PLSS_ERR_TIMEOUT = -5,    /* the iteration driver ran more bodies than  */
                              /* 2 (maxit + 2) + 8 allow (a safety bound)  */
    PLSS_ERR_BUSY = -6,       /* server queue full / admission refused      */
    PLSS_ERR_NOT_FOUND = -7   /* unknown ticket                             */
} plss_status;

/* Sketches: RESIDUAL (Sec. 4, Algorithm 1), IDENTITY (Sec. 7), GENERAL
 * (Sec. 2.4: column k of S has entry i = -1 where bit 63 of output k*m + i
 * of the SplitMix64 stream seeded with plss_opts.seed is set, else +1; the
 * history of directions is capped at plss_opts.kacz_hist <= 1,024 and
 * emptied when full; maxit caps the columns drawn; W = I). */
enum { PLSS_SKETCH_RESIDUAL = 0, PLSS_SKETCH_IDENTITY = 1, PLSS_SKETCH_GENERAL = 2 };
/* PLSS_FP64: A, vectors and sums in double.
 * PLSS_FP32: A and the vectors r, p, W y stored as float, sums of products
 * accumulated in float; inner products, the scalar recursion, x and a
 * periodic true residual b - A x (refinement) in double. */
enum { PLSS_FP64 = 0, PLSS_FP32 = 1 };
/* Diagonal weight W of Sec. 4.1: identity, 1/||A_{:,j}||, 1/||A_{:,j}||^2
 * (an empty column gets weight 1). */
enum { PLSS_W_IDENTITY = 0, PLSS_W_COLNORM = 1, PLSS_W_COLNORM2 = 2 };

/* Storage of the sweeps (plss_create, plss_server_create). AUTO: tiles of
 * short rows (columns) whose padding stays within 1/4 are also stored
 * sliced -- 32 lanes side by side, so that a warp reads 32 consecutive
 * indices and values per load and g lanes sum one row (column) -- at the
 * cost of a second copy of those nonzeros; other tiles use the CSR (CSC).
 * CSR: the CSR and CSC only. A server with the CSR layout gives each request
 * the results of a context created with it (GRID schedule); with AUTO, the
 * results of the same request served alone. */
enum { PLSS_LAYOUT_AUTO = 0, PLSS_LAYOUT_CSR = 1 };

/* Schedule of a residual-sketch solve. GRID: every sweep is a grid-wide
 * kernel over all systems of the context. SMALL: when every system has at
 * most 2^20 nonzeros, one thread-block cluster of 8 CTAs per system runs
 * whole iterations, its CTAs meeting at cluster barriers and exchanging
 * partial sums through distributed shared memory (no kernel boundaries
 * between the sweeps; plss_kernel_times then records nothing); when the
 * largest system's m + n vector entries take at most 128 KB in the storage
 * type, every CTA also keeps copies of r and p in its shared memory for the
 * sweeps' gathers (same arithmetic); otherwise as GRID. AUTO: SMALL when it fits and every system has at most 65,536
 * nonzeros or the systems are at least 1/8 as many as the SMs; else GRID.
 * The schedules reduce in different orders: their iterates agree to
 * rounding, not bit for bit. */
enum { PLSS_SCHED_AUTO = 0, PLSS_SCHED_GRID = 1, PLSS_SCHED_SMALL = 2, PLSS_SCHED_COOP = 3 };
/* COOP: for a single-system context whose rows and columns are both sliced
 * throughout (plss_ctx_layout), whole iterations run in one cooperative
 * launch over the GPU (the sweeps and the update as phases that meet at
 * grid barriers, every CTA taking the scalar steps on its own copy of the
 * state); any other context runs as AUTO. A grid barrier that waits longer
 * than 2 s ends the solve with PLSS_ERR_TIMEOUT. No per-kernel timings
 * (plss_kernel_times records nothing). */

/* A sparse matrix in CSR form (see the conventions above). val holds nnz
 * doubles, or floats when val_f32 = 1. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const void *val;
    int32_t val_f32;
    int32_t on_device;
} plss_csr;

/* Options. Call plss_opts_default() first, then override fields. */
typedef struct {
    int32_t sketch;         /* PLSS_SKETCH_*                                        */
    int32_t precision;      /* PLSS_FP64 / PLSS_FP32 (fixed at create: storage)     */
    int32_t w_mode;         /* PLSS_W_*                                             */
    int32_t stop_on_true;   /* 1: stop only when b - A x (recomputed in double)     */
                            /*    passes the test; forced to 1 for PLSS_FP32       */
    double tol;             /* stop when ||r||/||b|| <= tol (Sec. 5)                */
    int64_t maxit;          /* cap on updates (residual) or rows visited (identity);*/
                            /* < 0 means n                                          */
    int64_t refine_period;  /* PLSS_FP32: also restart from b - A x every this many */
                            /* updates (<= 0: off)                                 */
    int64_t kacz_hist;      /* identity sketch: history window K (0 = Kaczmarz,    */
                            /* <= 64 per system, <= 4,096 for one system);         */
                            /* general sketch: history of directions (<= 1,024)    */
    uint64_t seed;          /* identity sketch: row-order stream seed; general     */
                            /* sketch: sketch-column stream seed                   */
    int32_t io_device;      /* 1: b, x0, x_out are device pointers                  */
    int32_t symmetric;      /* create: caller asserts A^T = A (square); A^T r then  */
                            /* reuses the CSR and no transpose is stored           */
    void *stream;           /* cudaStream_t to run on (NULL: the legacy stream)     */
    double *hist;           /* optional host array [hist_cap][5]: for update k+1 of */
                            /* system 0, (rho_k, phi_{k+1}, beta_k, gamma_k,        */
                            /* theta_{k+1}) -- the scalars of Algorithm 1          */
    int64_t hist_cap;
    int32_t profile;        /* 1: time every sweep launch with CUDA events recorded */
                            /* on the solve's stream (see plss_kernel_times);      */
                            /* k > 1: time one chunk of launches in k             */
    int32_t layout;         /* create: PLSS_LAYOUT_* (storage of the sweeps' tiles) */
    double inner_tol;       /* PLSS_FP32: restart from b - A x (refinement) once   */
                            /* the recursive residual has fallen by this factor    */
                            /* since the last start (default 1e-4; 0 = off)        */
    int32_t schedule;       /* residual sketch: PLSS_SCHED_* (how the iterations   */
                            /* are spread over the GPU)                           */
    int32_t tile_shift;     /* create: sweep tiles of 2^tile_shift times the       */
                            /* default nonzeros, -2..2 (0 = default; the knob     */
                            /* plss_tune measures)                                */
    int32_t refine_mode;    /* residual sketch: PLSS_REFINE_* (what a refresh of  */
                            /* the residual from b - A x does)                    */
} plss_opts;

/* Refinement modes of the residual sketch (an extension, not in the paper).
 * A refresh recomputes r = b - A x in double: every refine_period updates,
 * when the recursive residual has fallen by inner_tol (FP32 storage), and
 * when a stop is confirmed false on b - A x (stop_on_true). RESTART: the
 * recursion starts anew from the fresh residual (a first step p = (rho/phi)
 * W y). REPLACE: the fresh residual replaces the recursive one and the
 * recursion goes on with its p and theta (residual replacement; in exact
 * arithmetic nothing changes); it also applies refine_period in FP64
 * storage. A breakdown always restarts. Single and batched residual-sketch
 * solves; plss_solve_rhs and the server use RESTART. */
enum { PLSS_REFINE_RESTART = 0, PLSS_REFINE_REPLACE = 1 };

/* Outcome of one solve. relres_rec is sqrt(rho)/||b|| of the last recursive
 * (or refined) residual; relres_true is ||b - A x||/||b|| recomputed in
 * double after the solve; seconds is device time between the solve's first
 * and last kernel. */
typedef struct {
    int32_t status;
    int32_t reserved;
    int64_t iters;
    double relres_rec;
    double relres_true;
    double seconds;
} plss_result;

typedef struct plss_ctx plss_ctx;

void plss_opts_default(plss_opts *o);

/* The problem of the paper's Sec. 1: A x = b with A in R^{m x n} of any
 * shape and rank and b in range(A) (a consistent system); a context holds
 * one such A for any number of solves with it.
 * Copies A to the device, validates it, builds its transpose (unless
 * o->symmetric) and the tile schedule of the sparse sweeps (o->layout,
 * o->tile_shift). The storage precision is o->precision. A malformed CSR,
 * an unknown precision or layout, or tile_shift outside [-2, 2] returns
 * PLSS_ERR_INVALID with nothing allocated on the device. On error *out is
 * NULL. */
plss_status plss_create(const plss_csr *A, const plss_opts *o, plss_ctx **out);

/* As plss_create for nsys independent systems As[0..nsys-1], packed into one
 * block-diagonal context so that every sweep covers all systems in one
 * launch while scalars, stopping and status stay per system. Each system
 * runs the paper's Algorithm 1 on its own; solving many systems at once has
 * no counterpart in the paper. */
plss_status plss_create_batched(const plss_csr *As, int32_t nsys, const plss_opts *o,
                                plss_ctx **out);

/* Frees the context and all device memory it owns; NULL is ignored. */
void plss_destroy(plss_ctx *ctx);

/* One candidate plan measured by plss_tune. */
typedef struct {
    int32_t layout;         /* PLSS_LAYOUT_*                                        */
    int32_t tile_shift;     /* as in plss_opts                                      */
    int32_t schedule;       /* PLSS_SCHED_GRID or PLSS_SCHED_SMALL                  */
    int32_t status;         /* PLSS_OK, or the error that ruled the candidate out   */
    double us_per_update;   /* wall time of the timed solve / its updates (0 if not */
                            /* measured)                                          */
} plss_tune_entry;

/*
 * Autotuner of the sweep plan (the paper has none: the plan is this library's).
 * For each candidate -- layout AUTO and CSR, tile_shift -1, 0 and 1, and
 * schedule GRID, plus SMALL where every system fits the cluster schedule --
 * it builds a context of As[0..nsys-1] with o's precision and symmetric flag,
 * computes the consistent right-hand sides b = A 1 on the device, runs one
 * untimed and one timed solve of exactly `updates` updates of the residual
 * sketch (tol 0, o's w_mode), and measures the timed one on the host clock
 * (wall time, launches and synchronisation included). Only one candidate
 * context exists at a time.
 *   best: *o with layout, tile_shift and schedule of the fastest candidate.
 *   entries[0 .. min(cap, *count)): every candidate in the order tried;
 *   *count = the number of candidates. entries may be NULL when cap is 0.
 * A candidate that cannot be built for lack of device memory is recorded
 * with PLSS_ERR_NOMEM and skipped; any other failure is returned.
 * PLSS_ERR_INVALID for NULL As/best/count, nsys <= 0, updates outside
 * [1, 100000], cap < 0, or entries NULL with cap > 0.
 */
plss_status plss_tune(const plss_csr *As, int32_t nsys, const plss_opts *o, int32_t updates,
                      plss_opts *best, plss_tune_entry *entries, int32_t cap, int32_t *count);

/* Sizes of a context: systems, total rows, total columns, total nonzeros. */
plss_status plss_ctx_info(const plss_ctx *ctx, int32_t *nsys, int64_t *m, int64_t *n,
                          int64_t *nnz);

/* Tile schedule of a context's sweeps (PLSS_LAYOUT_*; an inspection call
 * with no counterpart in the paper): out[0] row tiles, out[1] of them
 * sliced, out[2] column tiles, out[3] of them sliced, out[4] and out[5]
 * elements (nonzeros plus padding) of the sliced row and column copies.
 * PLSS_ERR_INVALID on a NULL argument. */
plss_status plss_ctx_layout(const plss_ctx *ctx, int64_t out[6]);

/*
 * Solves A x = b for a single-system context.
 *   b[m], x0[n] (NULL = zero start), x_out[n]: host, or device when
 *   o->io_device. The residual sketch runs Algorithm 1; the identity sketch
 *   runs eq:pkKacz with rows in a fresh SplitMix64/Fisher-Yates permutation
 *   per pass (seed o->seed) and tests ||b - A x|| after every pass; the
 *   general sketch draws one random sign column per step (Corollary 2.2)
 *   and tests ||b - A x|| before every step.
 * Returns PLSS_OK, PLSS_NOT_CONVERGED (x_out holds the last iterate), or
 * PLSS_ERR_BREAKDOWN when phi_1 <= 0 (A^T r_0 = 0 with r_0 != 0: b is not in
 * range(A)) or when (sqrt(theta phi)/rho - 1)(sqrt(theta phi)/rho + 1) <= 0,
 * which happens only when A^T r_k is parallel to p_k; x_out then holds the
 * last iterate. ||b|| = 0 returns x0 at once with PLSS_OK.
 */
plss_status plss_solve(plss_ctx *ctx, const double *b, const double *x0, double *x_out,
                       const plss_opts *o, plss_result *res);

/* Solves every system of a batched context at once (Algorithm 1 per
 * system, all systems' sweeps in the same launches): b[s], x0[s] (array of
 * NULL or NULL entries = zero start), x_out[s] for s < nsys; res[nsys].
 * Systems stop independently; the return value is PLSS_OK when all
 * converged, else the first non-OK system status. Residual sketch only. */
plss_status plss_solve_batched(plss_ctx *ctx, const double *const *b, const double *const *x0,
                               double *const *x_out, const plss_opts *o, plss_result *res);

/*
 * Checkpoint and resume of a residual-sketch solve (no counterpart in the
 * paper, whose whole iteration state -- Algorithm 1's x, r, p and the
 * scalars rho, theta and k -- is small enough to carry across a stop).
 *
 * A solve that the update cap (opts.maxit) stopped returns
 * PLSS_NOT_CONVERGED and leaves its state in the context: b, x, r, p, u = W y
 * and per system the scalars, the phase the recursion would have entered
 * next, the refinement counters and the update count. plss_resume goes on
 * from that state for every system the cap stopped, up to opts->maxit
 * updates in total (the count includes the updates already taken) and to
 * opts->tol; systems that converged or broke down are left as they are
 * (their x is still written to x_out). The iterates are the ones the
 * uninterrupted solve would have produced, bit for bit: every reduction
 * runs in a fixed order. opts must be the interrupted solve's (w_mode,
 * refine_period, inner_tol, refine_mode, stop_on_true) except maxit, tol,
 * stream, io_device, hist and hist_cap (the history of a resume starts at
 * row k of hist, k = the updates taken before); schedule may differ.
 * x_out[nsys] (entries may be NULL) and res[nsys] as in plss_solve_batched.
 * PLSS_ERR_INVALID when the context holds no such state (no residual-sketch
 * solve since it was created or loaded, or another sketch or plss_solve_rhs
 * ran since; they overwrite x and b).
 *
 * plss_state_save copies that state into a host buffer of
 * plss_state_bytes(ctx) bytes (a header, the per-system scalars, then b, x,
 * r, p, u in the context's storage type); plss_state_load copies it back
 * into a context built from the same matrices with the same precision and
 * layout of systems (checked: sizes, nonzero count, storage type; the
 * values of A are the caller's to keep equal), after which plss_resume
 * continues the saved solve. Both are synchronous (cudaMemcpy) and need no
 * solve in flight on the context. plss_state_bytes returns -1 for a NULL
 * context; save and load return PLSS_ERR_INVALID for a NULL argument or a
 * buffer shorter than plss_state_bytes, load also for a buffer from
 * another library version or another context shape, or whose per-system
 * scalars are not those of a finished solve (a phase other than finished,
 * a negative update count, a kept transition into no running phase). The
 * vectors are not checked: the buffer is otherwise trusted.
 */
plss_status plss_resume(plss_ctx *ctx, double *const *x_out, const plss_opts *o, plss_result *res);
int64_t plss_state_bytes(const plss_ctx *ctx);
plss_status plss_state_save(plss_ctx *ctx, void *buf, int64_t bytes);
plss_status plss_state_load(plss_ctx *ctx, const void *buf, int64_t bytes);

/* Many right-hand sides on one matrix (SpMM form; no counterpart in the
 * paper): B is m x nrhs, X0 and X are n x nrhs, all row-major double (X0 may
 * be NULL). Each column is an independent Algorithm 1 solve with its own
 * scalars, A p and A^T r taken for all columns in one sweep over A;
 * converged columns freeze.
 * res[nrhs]. Residual sketch only; 1 <= nrhs <= 32 (one warp lane per
 * column), else PLSS_ERR_INVALID. */
plss_status plss_solve_rhs(plss_ctx *ctx, int32_t nrhs, const double *B, const double *X0,
                           double *X, const plss_opts *o, plss_result *res);

/* One sparse product with the context's stored matrix in double -- the two
 * products of Algorithm 1 (A p and A^T r) as a service of their own:
 * transpose = 0: out[m] = A v[n]; transpose = 1: out[n] = A^T v[m].
 * v and out follow o->io_device. Single-system contexts. */
plss_status plss_spmv(plss_ctx *ctx, int32_t transpose, const double *v, double *out,
                      const plss_opts *o);

/* r = b - A x and *norm2 = ||r||^2 for callers that cannot allocate device
 * memory. The paper has no counterpart: this is a service of the library.
 * Who needs it: code that has handed the whole GPU to its own memory pool
 * (a framework's caching allocator or arena, where a library cudaMalloc would
 * fail or fragment the pool), or a latency-critical loop that fixes its
 * memory at start-up and forbids allocation afterwards. Every other entry
 * point allocates its workspace in plss_create / plss_server_create; this
 * one allocates nothing, on the device or the host: its scratch (one partial
 * sum per block of 1,024 rows, an arrival counter and an invalid-input flag)
 * is a static device array of about 33 KB that every GPU loading the library
 * holds until the process exits. It runs a row-group kernel of its own, so
 * its r and *norm2 agree with b - plss_spmv(A, x) to rounding, not bit for
 * bit.
 *   A: CSR with row_ptr int64 [m+1], col_idx int32 [nnz], val double [nnz];
 *   x double [n], b double [m], r double [m] (output), norm2 one double
 *   (output) -- all device memory of the current device (or managed
 *   memory), owned by the caller; another GPU's memory is refused.
 *   m <= 4,194,304 rows (the scratch capacity); larger m returns
 *   PLSS_ERR_INVALID without launching anything. m = 0 gives *norm2 = 0.
 * The CSR's contents are not checked on the host (that would need a copy):
 * the kernel skips a row whose [row_ptr[i], row_ptr[i+1]) is not inside
 * [0, nnz] and every entry whose column is outside [0, n), so it never reads
 * out of bounds, and then sets *norm2 to NaN to say the input broke the
 * contract (r is then meaningless).
 * The call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 * stream): r and *norm2 are valid once the stream reaches that point. The
 * first call on a device looks up the scratch's device address (once per
 * device, in the device's primary context; the cached address does not
 * survive a cudaDeviceReset); make that first call before any stream
 * capture. All calls share the one scratch array: calls whose kernels
 * overlap on the GPU (different streams, no ordering between them) race and
 * give wrong sums; the arrival counter and the flag are cleared on the
 * stream before each launch. */
plss_status plss_residual_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                                  const int32_t *col_idx, const double *val, const double *x,
                                  const double *b, double *r, double *norm2, void *stream);

/* Device time of the residual-sketch sweeps accumulated over the solves of
 * this context that ran with o->profile = k > 0 (GRID schedule): ms[0..2] =
 * total milliseconds of the row sweep (r = r - A p, rho), the column sweep
 * (y = A^T r, phi, scalar step) and the update (p, theta, x), between CUDA
 * events recorded around each kernel of one graph launch in k, over the
 * launches in which a system stayed active throughout; launches[0..2] = the
 * kernel launches those totals cover; launches[3] = every kernel the
 * profiled solves launched. reset = 1 clears the totals after reading.
 * Either array may be NULL (ms has 3 entries, launches 4). A diagnostic
 * with no counterpart in the paper. */
plss_status plss_kernel_times(plss_ctx *ctx, double *ms, int64_t *launches, int32_t reset);

/* The gather floor of a sweep, measured on the device: a kernel that walks
 * the sweep's own sliced index stream with the sweep's grid and warp ranges
 * and gathers the sweep's dense vector (side 0: the row sweep's p, one
 * entry per nonzero of A p; side 1: the column sweep's r, one per nonzero
 * of A^T r) and does nothing else. Each of `reps` timed runs (1..1000) is
 * preceded by a write of 256 MB that evicts L2 and a read of the vector
 * (which the solve finds in L2, just written); *us_median and *us_min
 * (either may be NULL) receive the device times in microseconds between
 * CUDA events around the kernel. The contents of p and r are read, not
 * changed. Single-system contexts whose side is sliced throughout
 * (plss_ctx_layout reports it); otherwise PLSS_ERR_INVALID. A diagnostic
 * with no counterpart in the paper: every nonzero of Algorithm 1's A p and
 * A^T r is one such gather, and on GB300 their rate, not HBM bytes, bounds
 * the sweeps. Allocates and frees 256 MB for the eviction. */
plss_status plss_gather_bound(plss_ctx *ctx, int32_t side, int32_t reps, double *us_median, double *us_min);

/* Message of the last error on the calling thread ("" when none). */
const char *plss_last_error(void);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of independent solves (no counterpart  */
/* in the paper; every request is an Algorithm 1 solve of its own)     */
/* ------------------------------------------------------------------ */

typedef struct plss_server plss_server;

typedef struct {
    int32_t max_slots;        /* systems resident on the device at once          */
    int32_t max_queue;        /* pending requests before plss_submit says BUSY   */
    int64_t hbm_budget_bytes; /* device arena for matrices and vectors; <= 0:    */
                              /* 4 GiB, capped at 80% of free memory             */
    int32_t precision;        /* PLSS_FP64 / PLSS_FP32 for every request         */
    int32_t bodies_per_poll;  /* iterations run between admission rounds (8)     */
    int32_t layout;           /* PLSS_LAYOUT_CSR (default) or PLSS_LAYOUT_AUTO   */
                              /* (sliced tiles, one lane per segment; measured   */
                              /* slower for serving: mixed batches of tiles)     */
    int32_t reserved;
} plss_server_opts;

void plss_server_opts_default(plss_server_opts *o);

/* Starts a server: one host thread owns a device arena sized by the budget
 * and runs every admitted system together -- each sweep of Algorithm 1 is
 * one launch over the tiles of all resident systems (continuous batching).
 * Between rounds of bodies_per_poll iterations it retires finished systems
 * (freeing their slot and arena ranges) and admits queued requests, in
 * arrival order, while a slot and arena room for the request's matrix,
 * transpose and vectors are free. */
plss_status plss_server_create(const plss_server_opts *so, plss_server **out);

/* Queues one solve. A, b (length A->m) and x0 (length A->n, or NULL) are host
 * arrays, copied before the call returns. o gives tol, maxit and w_mode
 * (residual sketch; the server always verifies convergence on b - A x).
 * *ticket identifies the request. PLSS_ERR_BUSY when the queue is full or
 * the request can never fit the arena; PLSS_ERR_INVALID for a malformed
 * request. Thread-safe. */
plss_status plss_submit(plss_server *srv, const plss_csr *A, const double *b, const double *x0,
                        const plss_opts *o, uint64_t *ticket);

/* Never blocks. PLSS_PENDING while the request is queued or running; once
 * finished, copies x (length n) to the host array x_out (may be NULL), fills
 * *res (may be NULL; res->seconds = submit-to-completion wall time) and
 * forgets the ticket, returning the solve's status. PLSS_ERR_NOT_FOUND for
 * an unknown or already collected ticket. Thread-safe. */
plss_status plss_poll(plss_server *srv, uint64_t ticket, double *x_out, plss_result *res);

/* Counters: completed requests, queued, running, arena bytes in use. */
plss_status plss_server_stats(plss_server *srv, int64_t *completed, int64_t *queued,
                              int64_t *running, int64_t *bytes_in_use);

/* Stops the server thread (pending and running requests are dropped) and
 * frees its device memory. */
void plss_server_destroy(plss_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* PLSS_H */
