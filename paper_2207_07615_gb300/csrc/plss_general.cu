// plss_general.cu -- PLSS with a general sketch (Sec. 2.4) on the GPU.
//
// The sketch S_k = [s_1 ... s_k] (eq:genS) grows by one random sign column
// per step; column k has entry i = -1 where bit 63 of output k*m + i of the
// SplitMix64 stream seeded with `seed` is set, else +1, so every entry is
// computed where it is needed from (seed, k, i) and no sketch is stored.
// The update of Corollary 2.2 is
//   p_k = (s_k^T r_{k-1} / delta_k) (y_k - Y_{k-1} N_{k-1} Y_{k-1}^T y_k),
//   y_k = A^T s_k,  delta_k = y_k^T y_k - y_k^T Y_{k-1} N_{k-1} Y_{k-1}^T y_k.
// Y_{k-1} N_{k-1} Y_{k-1}^T is the orthogonal projector onto span(Y_{k-1}),
// which is also span(p_1 ... p_{k-1}) with the p_j mutually orthogonal
// (Sec. 2.1). The GPU keeps that projector as the directions
// q_j = y_j - (projection of y_j on the earlier ones), Theta = diag(||q_j||^2):
//   c = Q^T y,  delta = y^T y - sum_j c_j^2 / theta_j,
//   q = y - Q Theta^{-1} c,  p = (s^T r / delta) q,
// the same numbers as Theorem 2.1's recursion for N without a k x k matrix:
// each step streams the history Q (n x nh, one direction per column, column
// j contiguous) twice, as two GEMVs spread over the whole GPU. The history
// holds at most K directions and is emptied when full, as the oracle does.
//
// One step is five grid kernels, the kernel boundaries ordering them:
//   g_rows     r = b - A x (CSR, x gathered), partials of ||r||^2 and s_k^T r;
//              block 0 first folds the previous step's theta partials
//              (theta of the last direction; nh += 1) and empties a full
//              history
//   g_cols     y = A^T s_k (CSC, s_k from the hash: no gather), ||y||^2 partials
//   g_qty      partials of c = Q^T y over column chunks of 8,192
//   g_decide   one CTA: stop test on ||r||, c, d = c / theta, delta, gamma,
//              the skip test
//   g_update   q = y - Q d, column nh of Q, x += gamma q, theta partials
// The host launches bodies of steps and reads the stop flag between them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plss.h"
#include "plss_ctx.h"
#include "plss_dev.cuh"
#include "plss_devfn.cuh"
#include "plss_launch.h"
#include "plss_trace.h"

namespace plss {

#define GS_TRY(expr)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return fail(PLSS_ERR_CUDA, "general sketch: %s: %s", #expr, cudaGetErrorString(e_)); \
        }                                                                                     \
    } while (0)

constexpr int kGsThreads = 256;
constexpr int kGsWarps = kGsThreads / 32;
constexpr int kGsMaxK = 1024;
constexpr int64_t kGsChunk = 8192;   // columns per partial dot product of c = Q^T y

struct GsState {
    double rr;        // ||r_{k-1}||^2 of the last g_rows
    double nb2;       // ||b||^2
    double tol;
    double gamma;     // step of the current column
    int64_t k;        // sketch columns drawn
    int64_t maxit;
    int64_t skipped;
    int32_t nh;       // directions in the history
    int32_t store;    // the last g_update produced a direction to keep
    int32_t done;     // 0 running, 1 converged, 2 column cap reached
    int32_t skip;     // this column is skipped (delta at rounding level)
};

struct GsArgs {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *val;
    const int32_t *col_ptr;
    const int32_t *row_idx;
    const void *cval;
    const double *b;
    double *x;
    double *r;
    double *y;
    double *Q;         // [K][n]
    double *theta;     // [K]
    double *d;         // [K]: c_j, then c_j / theta_j
    double *part_r;    // [2 * grid]: ||r||^2, s^T r
    double *part_y;    // [grid]
    double *part_c;    // [K * nch]: partial c_j over column chunk ch at j * nch + ch
    double *part_t;    // [grid]
    GsState *st;
    int64_t m, n;
    uint64_t seed;
    int32_t K, grid, nch;
    Sliced csl;   // the context's sliced columns with their warp ranges, or wr = null
    int32_t csl_grid, pad;   // the grid those warp ranges were cut for (<= grid)
};

struct GeneralState {
    int32_t K = -1;
    int32_t grid = 0;
    double *d_Q = nullptr, *d_theta = nullptr, *d_d = nullptr, *d_y = nullptr, *d_r = nullptr;
    double *d_part = nullptr;
    GsState *d_st = nullptr;
    GsState *h_st = nullptr;   // pinned
    // the body of kGsBody sketch columns captured as a CUDA graph for the
    // arguments it was captured with
    cudaGraphExec_t body = nullptr;
    GsArgs body_args{};
    int body_gr = 0, body_gc = 0;
    bool body_f32 = false;
};

// Sign of sketch entry (k, i): bit 63 of SplitMix64 output k*m + i.
__device__ __forceinline__ double gs_sign(uint64_t seed, int64_t m, int64_t k, int64_t i) {
    uint64_t z = seed + (uint64_t(k) * uint64_t(m) + uint64_t(i) + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (z >> 63) ? -1.0 : 1.0;
}

// Fixed-order CTA sum; the result is valid in thread 0.
__device__ __forceinline__ double gs_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kGsWarps; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Contiguous share [lo, hi) of `len` items for this CTA.
__device__ __forceinline__ void gs_range(int64_t len, int64_t &lo, int64_t &hi) {
    lo = len * int64_t(blockIdx.x) / int64_t(gridDim.x);
    hi = len * int64_t(blockIdx.x + 1) / int64_t(gridDim.x);
}

// Dot product of segment [s, e) of (idx, val) with a vector fetched by
// `get` (a gather of x, or the sketch sign of a row), split over the G
// lanes of a group: every lane issues 8 index/value loads, then its 8
// fetches, then its 8 FMAs; the sum lands in every lane of the group.
template <int G, typename S, typename F>
__device__ __forceinline__ double gs_dot(const int32_t *__restrict__ idx, const S *__restrict__ val, int32_t s,
                                         int32_t e, int gl, F &&get) {
    double acc = 0.0;
    for (int32_t base = s + gl; base < e; base += 8 * G) {
        int32_t c[8];
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int32_t q = base + u * G;
            const bool in = q < e;
            c[u] = in ? __ldg(idx + q) : 0;
            v[u] = in ? double(__ldg(val + q)) : 0.0;
        }
        double g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) g[u] = base + u * G < e ? get(c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fma(v[u], g[u], acc);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Calls body(seg, d) for the segments [lo, hi) of ptr, G lanes each (d the
// group's dot product, in the group's first lane); warp-uniform loop.
template <int G, typename S, typename F, typename B>
__device__ __forceinline__ void gs_segments(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                            const S *__restrict__ val, int64_t lo, int64_t hi, F &&get, B &&body) {
    constexpr int SPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane & (G - 1);
    for (int64_t base = lo + int64_t(warp) * SPW; base < hi; base += int64_t(kGsWarps) * SPW) {
        const int64_t seg = base + gid;
        const bool valid = seg < hi;
        const int32_t s0 = valid ? __ldg(ptr + seg) : 0, s1 = valid ? __ldg(ptr + seg + 1) : 0;
        const double d = gs_dot<G, S>(idx, val, s0, s1, gl, get);
        if (valid && gl == 0) body(seg, d);
    }
}

template <int G, typename S>
__global__ void __launch_bounds__(kGsThreads) g_rows(GsArgs a) {
    __shared__ double sh[kGsWarps];
    wait_prior_grid();
    GsState *st = a.st;
    if (st->done) return;
    if (blockIdx.x == 0 && st->store) {
        // the previous column's direction: theta = ||q||^2 over the CTAs'
        // partials in a fixed order
        double th = 0.0;
        for (int g = threadIdx.x; g < a.grid; g += kGsThreads) th += a.part_t[g];
        th = gs_sum(th, sh);
        if (threadIdx.x == 0) {
            if (th > 0.0) {
                a.theta[st->nh] = th;
                st->nh += 1;
            }
            st->store = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.K > 0 && st->nh == a.K) st->nh = 0;   // history full: start anew
    int64_t lo, hi;
    gs_range(a.m, lo, hi);
    const int64_t k = st->k;
    double rr = 0.0, sr = 0.0;
    const double *__restrict__ x = a.x;
    gs_segments<G, S>(a.row_ptr, a.col_idx, static_cast<const S *>(a.val), lo, hi,
                      [&](int32_t c) { return __ldcg(x + c); },
                      [&](int64_t i, double d) {
                          const double ri = a.b[i] - d;
                          a.r[i] = ri;
                          rr = fma(ri, ri, rr);
                          sr = fma(gs_sign(a.seed, a.m, k, i), ri, sr);
                      });
    rr = gs_sum(rr, sh);
    sr = gs_sum(sr, sh);
    if (threadIdx.x == 0) {
        a.part_r[2 * blockIdx.x] = rr;
        a.part_r[2 * blockIdx.x + 1] = sr;
    }
}

// y = A^T s_k over the columns (CSC, or the CSR of a symmetric A); the
// sketch entry of row i is computed from (seed, k, i), nothing is gathered.
template <int G, typename S>
__global__ void __launch_bounds__(kGsThreads) g_cols(GsArgs a) {
    __shared__ double sh[kGsWarps];
    wait_prior_grid();
    const GsState *st = a.st;
    if (st->done) return;
    int64_t lo, hi;
    gs_range(a.n, lo, hi);
    const int64_t k = st->k;
    const uint64_t seed = a.seed;
    const int64_t m = a.m;
    double yy = 0.0;
    gs_segments<G, S>(a.col_ptr, a.row_idx, static_cast<const S *>(a.cval), lo, hi,
                      [&](int32_t i) { return gs_sign(seed, m, k, i); },
                      [&](int64_t j, double d) {
                          a.y[j] = d;
                          yy = fma(d, d, yy);
                      });
    yy = gs_sum(yy, sh);
    if (threadIdx.x == 0) a.part_y[blockIdx.x] = yy;
}

// y = A^T s_k over the context's sliced columns (a single system whose
// columns are sliced throughout, warp ranges cut for this grid): the
// residual sketch's column-sweep walk -- 32 consecutive indices and values
// per warp load, 8 steps in flight -- with the sketch sign of each entry's
// row computed from its index in place of a gathered r.
template <typename S>
__global__ void __launch_bounds__(kGsThreads) g_cols_sliced(GsArgs a) {
    __shared__ double sh[kGsWarps];
    wait_prior_grid();
    const GsState *st = a.st;
    if (st->done) return;
    const int64_t k = st->k;
    const uint64_t seed = a.seed;
    const int64_t m = a.m;
    const int lane = threadIdx.x & 31;
    const int g = a.csl.g;
    const int32_t w = int32_t(threadIdx.x >> 5) * int32_t(gridDim.x) + int32_t(blockIdx.x);
    const int32_t s0 = __ldg(a.csl.wr + w), s1 = __ldg(a.csl.wr + w + 1);
    const int32_t *__restrict__ idx = a.csl.idx;
    const S *__restrict__ val = static_cast<const S *>(a.csl.val);
    double yy = 0.0;
    for (int32_t sl = s0; sl < s1; ++sl) {
        const int32_t off = __ldg(a.csl.ptr + sl);
        const int32_t width = (__ldg(a.csl.ptr + sl + 1) - off) >> 5;
        const int32_t col = __ldg(a.csl.seg + 32 * sl + lane);
        double d = 0.0;
        for (int32_t k0 = 0; k0 < width; k0 += 8) {
            int32_t c[8];
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool in = k0 + u < width;
                const int32_t e = off + 32 * (k0 + u) + lane;
                c[u] = in ? __ldg(idx + e) : -1;
                v[u] = in ? double(__ldg(val + e)) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) d = fma(v[u], c[u] >= 0 ? gs_sign(seed, m, k, c[u]) : 0.0, d);
        }
        for (int o = g >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (col >= 0 && (lane & (g - 1)) == 0) {
            a.y[col] = d;
            yy = fma(d, d, yy);
        }
    }
    yy = gs_sum(yy, sh);
    if (threadIdx.x == 0) a.part_y[blockIdx.x] = yy;
    // the decision sums `grid` partials: those past this launch's are zero
    if (blockIdx.x == 0)
        for (int32_t b = int32_t(gridDim.x) + int32_t(threadIdx.x); b < a.grid; b += kGsThreads) a.part_y[b] = 0.0;
}

// Lanes per segment for a mean segment length: the largest power of two G
// <= 32 with 8 G <= the mean (each lane then has at least 8 entries).
static int gs_lanes(int64_t nnz, int64_t segs) {
    int g = 1;
    while (g < 32 && 2 * g * 8 * std::max<int64_t>(segs, 1) <= nnz) g <<= 1;
    return g;
}

// The per-column kernels are launched with programmatic dependent launch
// (launch_pdl): each waits for its predecessor in wait_prior_grid() before
// reading anything, and the launch of the next overlaps the end of the last.
template <typename S>
static cudaError_t launch_rows(int G, int grid, cudaStream_t s, const GsArgs &a) {
    switch (G) {
        case 1: return launch_pdl(g_rows<1, S>, grid, s, a);
        case 2: return launch_pdl(g_rows<2, S>, grid, s, a);
        case 4: return launch_pdl(g_rows<4, S>, grid, s, a);
        case 8: return launch_pdl(g_rows<8, S>, grid, s, a);
        case 16: return launch_pdl(g_rows<16, S>, grid, s, a);
        default: return launch_pdl(g_rows<32, S>, grid, s, a);
    }
}

template <typename S>
static cudaError_t launch_cols(int G, int grid, cudaStream_t s, const GsArgs &a) {
    switch (G) {
        case 1: return launch_pdl(g_cols<1, S>, grid, s, a);
        case 2: return launch_pdl(g_cols<2, S>, grid, s, a);
        case 4: return launch_pdl(g_cols<4, S>, grid, s, a);
        case 8: return launch_pdl(g_cols<8, S>, grid, s, a);
        case 16: return launch_pdl(g_cols<16, S>, grid, s, a);
        default: return launch_pdl(g_cols<32, S>, grid, s, a);
    }
}


// c_j = q_j^T y as partial dot products over column chunks: item (j, ch)
// sums chunk ch of direction j (coalesced over the chunk) into
// part_c[j * nch + ch]; the CTAs take items in turn.
__global__ void __launch_bounds__(kGsThreads) g_qty(GsArgs a) {
    __shared__ double sh[kGsWarps];
    wait_prior_grid();
    const GsState *st = a.st;
    if (st->done) return;
    const int64_t items = int64_t(st->nh) * a.nch;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t j = it / a.nch, ch = it % a.nch;
        const int64_t lo = ch * kGsChunk, hi = lo + kGsChunk < a.n ? lo + kGsChunk : a.n;
        const double *q = a.Q + j * a.n;
        double acc = 0.0;
        for (int64_t t = lo + threadIdx.x; t < hi; t += kGsThreads) acc = fma(q[t], a.y[t], acc);
        acc = gs_sum(acc, sh);
        if (threadIdx.x == 0) a.part_c[it] = acc;
    }
}

// One CTA: the stop test on r_{k-1}, then c, d, delta, gamma for column k.
__global__ void __launch_bounds__(kGsThreads) g_decide(GsArgs a) {
    __shared__ double sh[kGsWarps];
    __shared__ int sh_go;
    wait_prior_grid();
    GsState *st = a.st;
    if (st->done) return;
    double rr = 0.0, sr = 0.0, yy = 0.0;
    for (int g = threadIdx.x; g < a.grid; g += kGsThreads) {
        rr += a.part_r[2 * g];
        sr += a.part_r[2 * g + 1];
        yy += a.part_y[g];
    }
    rr = gs_sum(rr, sh);
    sr = gs_sum(sr, sh);
    yy = gs_sum(yy, sh);
    if (threadIdx.x == 0) {
        st->rr = rr;
        int go = 1;
        if (st->nb2 == 0.0 || sqrt(rr) <= st->tol * sqrt(st->nb2)) {
            st->done = 1;
            go = 0;
        } else if (st->k >= st->maxit) {
            st->done = 2;
            go = 0;
        }
        sh_go = go;
    }
    __syncthreads();
    if (!sh_go) return;
    const int nh = st->nh;
    // c_j = sum over CTAs of the partials (CTA order), d_j = c_j / theta_j
    double d2 = 0.0;
    for (int j = threadIdx.x; j < nh; j += kGsThreads) {
        double c = 0.0;
        for (int ch = 0; ch < a.nch; ++ch) c += a.part_c[int64_t(j) * a.nch + ch];
        d2 += (c * c) / a.theta[j];
        a.d[j] = c / a.theta[j];
    }
    d2 = gs_sum(d2, sh);
    if (threadIdx.x == 0) {
        const double ny = sqrt(yy), nd = sqrt(d2);
        const double delta = (ny - nd) * (ny + nd);
        st->skip = !(delta > 1e-14 * yy) ? 1 : 0;
        st->gamma = st->skip ? 0.0 : sr / delta;
        if (st->skip) st->skipped += 1;
        st->k += 1;
    }
}

// q = y - Q d on this CTA's column range: column nh of Q (when the history
// keeps directions), x += gamma q, theta partial.
__global__ void __launch_bounds__(kGsThreads) g_update(GsArgs a) {
    __shared__ double sh[kGsWarps];
    __shared__ double sd[kGsMaxK];
    wait_prior_grid();
    GsState *st = a.st;
    if (st->done || st->skip) return;
    const int nh = st->nh;
    const double gamma = st->gamma;
    for (int j = threadIdx.x; j < nh; j += kGsThreads) sd[j] = a.d[j];
    __syncthreads();
    int64_t lo, hi;
    gs_range(a.n, lo, hi);
    double tq = 0.0;
    for (int64_t t = lo + threadIdx.x; t < hi; t += kGsThreads) {
        double q = a.y[t];
        for (int j = 0; j < nh; ++j) q -= a.Q[int64_t(j) * a.n + t] * sd[j];
        if (a.K > 0) a.Q[int64_t(nh) * a.n + t] = q;
        a.x[t] = __dadd_rn(a.x[t], __dmul_rn(gamma, q));
        tq = fma(q, q, tq);
    }
    tq = gs_sum(tq, sh);
    if (threadIdx.x == 0) a.part_t[blockIdx.x] = tq;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->store = a.K > 0 ? 1 : 0;
}

constexpr int64_t kGsBody = 16;   // sketch columns between reads of the stop flag

// One column: the five kernels in order.
static cudaError_t launch_column(bool f32, int gr, int gc, int grid, cudaStream_t s, const GsArgs &a) {
    cudaError_t e = f32 ? launch_rows<float>(gr, grid, s, a) : launch_rows<double>(gr, grid, s, a);
    if (e == cudaSuccess) {
        if (a.csl.wr)
            e = f32 ? launch_pdl(g_cols_sliced<float>, a.csl_grid, s, a) : launch_pdl(g_cols_sliced<double>, a.csl_grid, s, a);
        else e = f32 ? launch_cols<float>(gc, grid, s, a) : launch_cols<double>(gc, grid, s, a);
    }
    if (e == cudaSuccess) e = launch_pdl(g_qty, grid, s, a);
    if (e == cudaSuccess) e = launch_pdl(g_decide, 1, s, a);
    if (e == cudaSuccess) e = launch_pdl(g_update, grid, s, a);
    return e;
}

// ||v||^2 in two launches: one partial per CTA over its contiguous share,
// then one CTA sums the partials in CTA order.
__global__ void __launch_bounds__(kGsThreads) g_norm2_part(const double *v, int64_t len, double *part) {
    __shared__ double sh[kGsWarps];
    int64_t lo, hi;
    gs_range(len, lo, hi);
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kGsThreads) acc = fma(v[i], v[i], acc);
    acc = gs_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kGsThreads) g_norm2_sum(const double *part, int32_t np, double *out) {
    __shared__ double sh[kGsWarps];
    double acc = 0.0;
    for (int32_t g = threadIdx.x; g < np; g += kGsThreads) acc += part[g];
    acc = gs_sum(acc, sh);
    if (threadIdx.x == 0) *out = acc;
}

static void general_free(GeneralState *g) {
    if (!g) return;
    dfree(g->d_Q);
    dfree(g->d_theta);
    dfree(g->d_d);
    dfree(g->d_y);
    dfree(g->d_r);
    dfree(g->d_part);
    dfree(g->d_st);
    if (g->h_st) cudaFreeHost(g->h_st);
    if (g->body) cudaGraphExecDestroy(g->body);
    delete g;
}

void free_general(plss_ctx *c) {
    general_free(c->gen);
    c->gen = nullptr;
}

static plss_status general_prepare(plss_ctx *c, int32_t K) {
    if (c->gen && c->gen->K == K) return PLSS_OK;
    free_general(c);
    GeneralState *g = new GeneralState();
    g->K = K;
    g->grid = c->nsm * 4;
    const size_t Kc = size_t(std::max(K, 1));
    plss_status st = PLSS_OK;
    if ((st = dalloc(reinterpret_cast<void **>(&g->d_Q), 8 * Kc * size_t(std::max<int64_t>(c->n, 1)), "Q")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&g->d_theta), 8 * Kc, "theta")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&g->d_d), 8 * Kc, "d")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&g->d_y), 8 * size_t(std::max<int64_t>(c->n, 1)), "y")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&g->d_r), 8 * size_t(std::max<int64_t>(c->m, 1)), "r")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&g->d_part),
                     8 * (4 * size_t(g->grid) + Kc * size_t((std::max<int64_t>(c->n, 1) + kGsChunk - 1) / kGsChunk)),
                     "partials")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&g->d_st), sizeof(GsState), "state")) != PLSS_OK) {
        general_free(g);
        return st;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&g->h_st), sizeof(GsState)) != cudaSuccess) {
        general_free(g);
        return fail(PLSS_ERR_NOMEM, "pinned allocation failed");
    }
    c->gen = g;
    return PLSS_OK;
}

plss_status run_general(plss_ctx *c, const double *b, const double *x0, double *x_out, const plss_opts *o,
                        plss_result *res) {
    TraceRange tr("plss: solve (general sketch)");
    plss_status st = check_opts(o);
    if (st != PLSS_OK) return st;
    if (o->kacz_hist < 0 || o->kacz_hist > kGsMaxK)
        return fail(PLSS_ERR_INVALID, "the general sketch keeps a history of 0..%d directions (kacz_hist)", kGsMaxK);
    if (o->w_mode != PLSS_W_IDENTITY) return fail(PLSS_ERR_INVALID, "the general sketch takes W = I");
    c->state_valid = false;   // x and b of the context are overwritten: nothing to resume
    cudaStream_t s = static_cast<cudaStream_t>(o->stream);
    const bool dev = o->io_device != 0;
    const int32_t K = int32_t(o->kacz_hist);
    if ((st = general_prepare(c, K)) != PLSS_OK) return st;
    GeneralState *g = c->gen;
    if (c->m > 0 && !b) return fail(PLSS_ERR_INVALID, "b is NULL");
    if ((st = put_vec(c->d_b, b, c->m, dev, s)) != PLSS_OK) return st;
    if ((st = put_vec(c->d_x, x0, c->n, dev, s)) != PLSS_OK) return st;

    GsArgs a;
    std::memset(&a, 0, sizeof a);   // padding too: the body graph is keyed by these bytes
    a.row_ptr = c->d_row_ptr;
    a.col_idx = c->d_col_idx;
    a.val = c->d_val;
    a.col_ptr = c->d_col_ptr;
    a.row_idx = c->d_row_idx;
    a.cval = c->d_cval;
    a.b = c->d_b;
    a.x = c->d_x;
    a.r = g->d_r;
    a.y = g->d_y;
    a.Q = g->d_Q;
    a.theta = g->d_theta;
    a.d = g->d_d;
    a.part_r = g->d_part;
    a.part_y = g->d_part + 2 * g->grid;
    a.part_t = g->d_part + 3 * g->grid;
    a.part_c = g->d_part + 4 * g->grid;
    a.st = g->d_st;
    a.m = c->m;
    a.n = c->n;
    a.seed = o->seed;
    a.K = K;
    a.grid = g->grid;
    a.nch = int32_t((std::max<int64_t>(c->n, 1) + kGsChunk - 1) / kGsChunk);
    // the sliced columns, over the grid their warp ranges were cut for
    if (c->d_cwr && c->csl.wr && c->grid_c <= g->grid) {
        a.csl = c->csl;
        a.csl_grid = c->grid_c;
    }

    GsState z{};
    z.tol = o->tol;
    z.maxit = o->maxit < 0 ? c->n : o->maxit;
    *g->h_st = z;
    GS_TRY(cudaMemcpyAsync(g->d_st, g->h_st, sizeof(GsState), cudaMemcpyHostToDevice, s));
    g_norm2_part<<<g->grid, kGsThreads, 0, s>>>(c->d_b, c->m, g->d_part);
    g_norm2_sum<<<1, kGsThreads, 0, s>>>(g->d_part, g->grid, &g->d_st->nb2);
    GS_TRY(cudaEventRecord(c->ev0, s));
    const int grid = g->grid;
    const int gr = gs_lanes(c->nnz, c->m), gc = gs_lanes(c->nnz, c->n);
    const int64_t body = kGsBody;
    // the body of kGsBody columns as a CUDA graph, captured again only when
    // its arguments change (a new seed, tolerance-independent otherwise)
    if (!g->body || std::memcmp(&g->body_args, &a, sizeof a) != 0 || g->body_gr != gr || g->body_gc != gc ||
        g->body_f32 != c->f32) {
        if (g->body) cudaGraphExecDestroy(g->body);
        g->body = nullptr;
        cudaGraph_t graph = nullptr;
        GS_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int64_t q = 0; q < body && e == cudaSuccess; ++q) e = launch_column(c->f32, gr, gc, grid, c->cap_stream, a);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return fail(PLSS_ERR_CUDA, "general sketch: graph capture failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        const cudaError_t e3 = cudaGraphInstantiate(&g->body, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) {
            g->body = nullptr;
            cudaGetLastError();
            return fail(PLSS_ERR_CUDA, "general sketch: graph instantiate failed: %s", cudaGetErrorString(e3));
        }
        g->body_args = a;
        g->body_gr = gr;
        g->body_gc = gc;
        g->body_f32 = c->f32;
    }
    for (int64_t it = 0;; it += body) {
        GS_TRY(cudaGraphLaunch(g->body, s));
        GS_TRY(cudaMemcpyAsync(g->h_st, g->d_st, sizeof(GsState), cudaMemcpyDeviceToHost, s));
        GS_TRY(cudaStreamSynchronize(s));
        if (g->h_st->done) break;
        if (it > z.maxit + 2 * body) return fail(PLSS_ERR_TIMEOUT, "general sketch: step driver overran");
    }
    GS_TRY(cudaEventRecord(c->ev1, s));
    if ((st = get_vec(x_out, c->d_x, c->n, dev, s)) != PLSS_OK) return st;
    GS_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const GsState &h = *g->h_st;
    // the last g_rows formed r for the returned x (the stop test ran on it)
    const double nb = std::sqrt(h.nb2);
    const double rel = nb > 0.0 ? std::sqrt(h.rr) / nb : 0.0;
    const plss_status out = h.done == 1 ? PLSS_OK : PLSS_NOT_CONVERGED;
    if (res) {
        res->status = out;
        res->reserved = 0;
        res->iters = h.k;
        res->relres_rec = rel;
        res->relres_true = rel;
        res->seconds = double(ms) * 1e-3;
    }
    return out;
}

}  // namespace plss
