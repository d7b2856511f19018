// plss_dev.cuh -- data layout shared by the host driver and the sm_103a kernels.
//
// Every context is a block-diagonal packing of one or more independent
// systems (one system for plss_create). Rows, columns and nonzeros of all
// systems live in single device arrays; column indices are global, so a
// sweep never needs to know which system a nonzero belongs to. The work of
// each sweep is cut into tiles that never straddle two systems; the scalar
// reductions of Algorithm 1 (rho, phi, theta) are per-tile partial sums
// followed, in the last tile of a system to finish, by a fixed-order sum
// (deterministic for a given tile schedule) and the system's scalar step.
#pragma once

#include <cstdint>

namespace plss {

constexpr int kThreads = 256;          // threads per CTA of every sweep
constexpr int kWarps = kThreads / 32;

// One unit of sweep work: segments (rows for A p, columns for A^T r, vector
// entries for the update) [begin, end) of system `sys`. `group` is the number
// of lanes that share one segment (1..32, a power of two); 0 means the whole
// CTA works on the single segment of the tile (very long rows/columns). With
// kSliced set, the sweeps read the tile from its sliced copy (below) instead;
// with kStaged set, they stage its products in shared memory; the low bits
// still give the lane count for kernels that use the plain CSR/CSC
// (products, residual norms).
constexpr int32_t kSliced = 0x100;
constexpr int32_t kStaged = 0x200;   // products staged in shared memory (at most 2,048 nonzeros, 1,024 segments)
constexpr int32_t kGroupMask = 0xff;

// Sliced copy of a side (rows or columns) of A. A sliced tile's segments,
// sorted by decreasing length (ties by index), form slices of 32 / g
// segments with g lanes each (slots q g .. q g + g - 1 hold segment q);
// slice s is as wide as ceil(longest segment / g) and stores the segment's
// element k in lane q g + (k mod g) at ptr[s] + 32 (k / g) + lane, so a warp
// reads 32 consecutive indices (values) per load. Padding has index -1 and
// value 0.
struct Sliced {
    int32_t g;              // lanes per segment (power of two, 1..32)
    const int32_t *first;   // [tiles] first slice of each tile
    const int32_t *ptr;     // [slices + 1] element offsets (multiples of 32)
    const int32_t *seg;     // [32 * slices] segment of each slot, -1 if none
    const int32_t *idx;     // padded indices
    const void *val;        // padded values (storage type)
    // Single-system contexts whose every tile of this side is sliced: the
    // sweep's grid has one range of slices [wr[w], wr[w + 1]) per warp
    // (balanced by elements); warp k of CTA b takes range k * gridDim.x + b,
    // so each CTA's warps draw from all along the length-sorted slices;
    // null otherwise.
    const int32_t *wr;
};

struct Tile {
    int32_t sys;
    int32_t begin;
    int32_t end;
    int32_t group;
};

// Static description of one system inside the packed context.
struct SysDesc {
    int64_t row_off;   // first global row
    int64_t col_off;   // first global column
    int32_t m, n;
    int32_t rt_begin, rt_count;   // row-sweep tiles
    int32_t ct_begin, ct_count;   // column-sweep tiles
    int32_t vt_begin, vt_count;   // vector-update tiles
};

// Phases of one system's iteration (see the body order in plss_kernels.cu).
enum Phase : int32_t {
    PH_SETUP = 0,   // next row sweep forms r = b - A x in double
    PH_FIRST = 1,   // r is fresh: next update is p = (rho/phi) W y
    PH_RUN = 2,     // 1-step recursion of Theorem 4.1
    PH_DONE = 3     // finished; `status` holds the outcome
};

// Mutable per-system state, device resident.
struct SysState {
    double rho, phi, theta, beta, gamma;
    double nb;          // ||b||
    double tol;
    double relres_rec;  // sqrt(rho)/||b|| of the last row sweep
    int64_t iters;      // updates applied
    int64_t maxit;
    int64_t since;      // updates since the last (re)start
    int64_t refine;     // FP32 storage: restart period (0 = never)
    double rho0;        // rho at the last (re)start
    double inner_tol2;  // FP32 storage: restart once rho <= inner_tol2 * rho0 (0 = off)
    double *hist;       // optional device array [hist_cap][5]
    int64_t hist_cap;
    int32_t phase;
    int32_t status;     // plss_status once phase == PH_DONE
    int32_t stop_on_true;
    int32_t upd;        // update due in this body: 0 none, 1 p = beta p + gamma u, 2 p = gamma u (first)
    uint32_t cnt_row, cnt_col, cnt_upd;
    int32_t resume;     // set when the update cap stopped the system: the transition it would
                        // have taken (phase | 0x10 reset `since` | 0x20 clear restart_next | 0x100)
    int32_t replace;       // refinement mode: 0 a refresh restarts the recursion, 1 it replaces r
    int32_t restart_next;  // the next set-up row sweep begins a new recursion (solve start, breakdown)
};

// Arguments of the three residual-sketch sweeps (one struct for all).
struct SweepArgs {
    // CSR of A (row sweep) and CSC of A (column sweep; equal to the CSR
    // pointers when A is symmetric)
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *val;
    const int32_t *col_ptr;
    const int32_t *row_idx;
    const void *cval;
    // tile schedules
    const Tile *rtiles;
    const Tile *ctiles;
    const Tile *vtiles;
    int32_t n_rtiles, n_ctiles, n_vtiles, pad;
    const SysDesc *desc;
    SysState *st;
    double *part_row;    // [2 * n_rtiles]
    double *part_col;    // [n_ctiles]
    double *part_upd;    // [n_vtiles]
    int32_t *n_active;   // systems not yet PH_DONE
    // vectors: b, x in double; r, p, u (= W y) in the storage type
    const double *b;
    double *x;
    void *r;
    void *p;
    void *u;
    const double *w;     // W = diag(w) or nullptr for W = I
    const double *winv;  // 1/w (theta = p^T W^{-1} p), nullptr with w
    const float *wf;     // float copies for the FP32-storage sweeps
    const float *winvf;
    Sliced rsl;          // sliced rows (tiles of rtiles flagged kSliced)
    Sliced csl;          // sliced columns (tiles of ctiles flagged kSliced)
};

}  // namespace plss
