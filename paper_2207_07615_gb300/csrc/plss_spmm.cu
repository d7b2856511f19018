// plss_spmm.cu -- many right-hand sides on one matrix (SpMM form of the
// residual-sketch sweeps of Algorithm 1).
//
// With k right-hand sides the vectors become blocks R (m x k), P, U, X
// (n x k), stored row-major with a row stride of 32, so that one warp owns
// one matrix row and lane j owns right-hand side j: every nonzero a_ij is
// read once for all k columns and the gathered row P[col, :] is one
// coalesced 128/256-byte access. Each column keeps its own scalars (rho, phi,
// theta, beta, gamma), its own stopping test and its own phase; a finished
// column is frozen while the others go on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "plss.h"
#include "plss_ctx.h"
#include "plss_dev.cuh"
#include "plss_devfn.cuh"
#include "plss_launch.h"
#include "plss_trace.h"

namespace plss {

constexpr int kRhsMax = 32;        // columns per solve (one warp lane each)
constexpr int kRhsStride = 32;     // row stride of the blocks
constexpr int kRhsRowsPerTile = 128;

struct RhsArgs {
    const int32_t *row_ptr, *col_idx;
    const void *val;
    const int32_t *col_ptr, *row_idx;
    const void *cval;
    const Tile *rtiles, *ctiles, *vtiles;
    int32_t n_rtiles, n_ctiles, n_vtiles, k;
    int64_t m, n;
    SysState *st;        // [k]
    double *part;        // [max tiles][2][32]
    double *part_init;   // [max tiles][2][32], partials of k_rhs_row_init
    uint32_t *cnt;       // [3]
    int32_t *n_active;
    const double *B;     // m x 32
    double *X;           // n x 32
    float *dX;           // FP32 storage: n x 32 float sum of the updates since the last (re)start
    void *R, *P, *U;     // storage type, (m|n) x 32
    const double *w;
    const double *winv;
    const float *wf;     // float copies (FP32 storage)
    const float *winvf;
};

struct RhsState {
    int32_t k = 0;
    double *d_B = nullptr, *d_X = nullptr;
    float *d_dX = nullptr;   // FP32 storage only
    void *d_R = nullptr, *d_P = nullptr, *d_U = nullptr;
    double *d_part = nullptr;   // 2 x [max tiles][64]: sweeps, then the restart row sweep
    SysState *d_st = nullptr;
    SysState *h_st = nullptr;
    uint32_t *d_cnt = nullptr;
    int32_t *d_active = nullptr;
    int32_t *h_active = nullptr;
    Tile *d_rt = nullptr, *d_ct = nullptr, *d_vt = nullptr;
    int32_t n_rt = 0, n_ct = 0, n_vt = 0;
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<double> hbuf;
};

__device__ __forceinline__ double rhs_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rhs_fma(float a, float b, float c) { return fmaf(a, b, c); }

// Per-lane accumulator of a sum of squares / products: double for FP64
// storage, double-float (FP32 operations only) for FP32 storage, so the
// FP32 sweeps spend no FP64 operation per block entry.
template <typename S>
struct RhsAcc;
template <>
struct RhsAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x, double y) { v = fma(x, y, v); }
    __device__ __forceinline__ double get() const { return v; }
};
template <>
struct RhsAcc<float> {
    DF v = {0.0f, 0.0f};
    __device__ __forceinline__ void add(float x, float y) { v = df_add_prod(v, x, y); }
    __device__ __forceinline__ double get() const { return double(v.hi) + double(v.lo); }
};

// Lane `lane`'s entry of (A_seg . V) for one segment [s, e) of a sparse
// side (indices idx, values val) against a stride-32 block V: the warp
// loads 32 index/value pairs at a time (coalesced), broadcasts them by
// shuffle and keeps 8 gathered block rows in flight before their FMAs;
// products are summed in segment order. `on` masks the lanes that take
// part in the gathers (every lane takes part in the shuffles).
template <typename VT, typename XT, typename ACC>
__device__ __forceinline__ ACC rhs_dot(const int32_t *__restrict__ idx, const VT *__restrict__ val, int32_t s,
                                       int32_t e, const XT *__restrict__ V, int lane, bool on) {
    ACC d = ACC(0);
    for (int32_t q0 = s; q0 < e; q0 += 32) {
        const int32_t q = q0 + lane;
        const int32_t cq = q < e ? __ldg(idx + q) : 0;
        const VT vq = q < e ? __ldg(val + q) : VT(0);
        const int nq = e - q0 < 32 ? int(e - q0) : 32;
        for (int u0 = 0; u0 < nq; u0 += 8) {
            XT g[8];
            ACC v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = (u0 + u) & 31;
                const int32_t c = __shfl_sync(0xffffffffu, cq, j);
                v[u] = ACC(__shfl_sync(0xffffffffu, vq, j));
                g[u] = on && u0 + u < nq ? V[int64_t(c) * kRhsStride + lane] : XT(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u0 + u < nq) d = rhs_fma(v[u], ACC(g[u]), d);
        }
    }
    return d;
}

// A lane's share of a block row: V consecutive right-hand sides (16 bytes:
// 4 floats or 2 doubles), so L = 32 / V lanes cover one block row and a
// warp works on V matrix rows at once. Indices and values are loaded by the
// L lanes of a row group from the same address (one request), the gathered
// block row is one 16-byte load per lane, and each lane spends V FMAs per
// nonzero: a few instructions per nonzero instead of one warp per nonzero.
template <typename S>
struct RhsVec;
template <>
struct RhsVec<float> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void ld(const float *p, float (&o)[4]) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
    }
    __device__ __forceinline__ static void ld_rw(const float *p, float (&o)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
    }
    __device__ __forceinline__ static void st(float *p, const float (&o)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <>
struct RhsVec<double> {
    static constexpr int V = 2;
    __device__ __forceinline__ static void ld(const double *p, double (&o)[2]) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = t.x, o[1] = t.y;
    }
    __device__ __forceinline__ static void ld_rw(const double *p, double (&o)[2]) {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        o[0] = t.x, o[1] = t.y;
    }
    __device__ __forceinline__ static void st(double *p, const double (&o)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    }
};

// d[v] = sum over the segment [s, e) of val * Vb[idx][off + v] for the lane's
// V right-hand sides (off = its first one), in segment order, 8 gathers in
// flight. `len_max` is the longest segment among the warp's row groups
// (warp-uniform loop); `on` skips the gathers of a lane with nothing to do.
template <typename S>
__device__ __forceinline__ void rhs_vdot(const int32_t *__restrict__ idx, const S *__restrict__ val, int32_t s,
                                         int32_t len, int32_t len_max, const S *__restrict__ Vb, int off, bool on,
                                         S (&d)[RhsVec<S>::V]) {
    constexpr int V = RhsVec<S>::V;
#pragma unroll
    for (int v = 0; v < V; ++v) d[v] = S(0);
    for (int32_t q0 = 0; q0 < len_max; q0 += 8) {
        int32_t c[8];
        S w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool in = on && q0 + u < len;
            c[u] = in ? __ldg(idx + s + q0 + u) : -1;
            w[u] = in ? __ldg(val + s + q0 + u) : S(0);
        }
        S g[8][V];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (c[u] >= 0) RhsVec<S>::ld(Vb + int64_t(c[u]) * kRhsStride + off, g[u]);
            else {
#pragma unroll
                for (int v = 0; v < V; ++v) g[u][v] = S(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c[u] >= 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) d[v] = rhs_fma(w[u], g[u][v], d[v]);
            }
    }
}

// Per right-hand side j, the fixed-order sum over the CTA of the V-lane
// partials (vec[v] of row group `grp`, lane group `ll`) and of the
// lane-per-column partials (one[j] in lane j); result in out[j] (thread j).
template <int V>
__device__ __forceinline__ void rhs_cta_sum_v(const double (&vec)[V], double one, double *out) {
    constexpr int G = 32 / (32 / V) * kWarps;   // row groups per CTA
    __shared__ double shv[G][32];
    __shared__ double sho[kWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = 32 / V, grp = warp * V + lane / L, ll = lane % L;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V; ++v) shv[grp][ll * V + v] = vec[v];
    sho[warp][lane] = one;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int q = 0; q < G; ++q) t += shv[q][threadIdx.x];
        for (int w = 0; w < kWarps; ++w) t += sho[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// Per-lane sum over the CTA's warps (lane j = column j) into part[0..31]
// of the tile, fixed order.
__device__ __forceinline__ void rhs_cta_sum(double v0, double v1, double *out0, double *out1) {
    __shared__ double sh[2][kWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    sh[0][warp][lane] = v0;
    sh[1][warp][lane] = v1;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            s0 += sh[0][w][threadIdx.x];
            s1 += sh[1][w][threadIdx.x];
        }
        out0[threadIdx.x] = s0;
        if (out1) out1[threadIdx.x] = s1;
    }
}

// Last CTA of a sweep: sum the tiles' partials per column (fixed order);
// returns true in the CTA that does it, with sums in sh_out (per lane).
__device__ __forceinline__ bool rhs_arrive(uint32_t *cnt, int32_t ntiles) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(cnt, 1u) == uint32_t(ntiles - 1);
    }
    __syncthreads();
    const bool last = s_last != 0;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last CTA: per-column sum of the CTAs' partials (stride 64 doubles
// per CTA, column j at offset which*32 + j), in a fixed order; the result is
// valid in threads 0..31.
__device__ __forceinline__ void rhs_final_sums(const double *part, int32_t nparts, int which,
                                               double &out) {
    __shared__ double sh[kWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s = 0.0;
    for (int32_t t = warp; t < nparts; t += kWarps) s += __ldcg(part + int64_t(t) * 64 + which * 32 + lane);
    __syncthreads();
    sh[warp][lane] = s;
    __syncthreads();
    out = 0.0;
    if (threadIdx.x < 32)
        for (int w = 0; w < kWarps; ++w) out += sh[w][threadIdx.x];
}

__device__ __forceinline__ void rhs_done(const RhsArgs &a, SysState *st, int32_t status) {
    st->status = status;
    st->phase = PH_DONE;
    atomicSub(a.n_active, 1);
}

// Row sweep of the columns that (re)start: r = b - A x with products in
// double, lane-per-column form; per-CTA partials of rho and ||b||^2 in
// part_init for k_rhs_row (launched next with the same grid) to finish.
// Returns at once when no column restarts (the usual case).
template <typename S>
__global__ void __launch_bounds__(kThreads) k_rhs_row_init(RhsArgs a) {
    wait_prior_grid();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool mine = lane < a.k;
    const int32_t ph = mine ? *reinterpret_cast<const volatile int32_t *>(&a.st[lane].phase) : PH_DONE;
    const bool init = ph == PH_SETUP;
    const bool any_init = __any_sync(0xffffffffu, init);
    if (!any_init) return;   // uniform: every warp reads the same phases
    const S *val = static_cast<const S *>(a.val);
    S *R = static_cast<S *>(a.R);
    double acc_i = 0.0, acc_b = 0.0;
    for (int32_t ti = blockIdx.x; ti < a.n_rtiles; ti += gridDim.x) {
        const Tile t = a.rtiles[ti];
        for (int32_t row = t.begin + warp; row < t.end; row += kWarps) {
            const int32_t s = a.row_ptr[row], e = a.row_ptr[row + 1];
            const int64_t ix = int64_t(row) * kRhsStride + lane;
            const double bi = init ? a.B[ix] : 0.0;
            double d = rhs_dot<S, double, double>(a.col_idx, val, s, e, a.X, lane, init);
            if (a.dX) d += rhs_dot<S, float, double>(a.col_idx, val, s, e, a.dX, lane, init);
            if (init) {
                const S ri = S(bi - d);
                R[ix] = ri;
                acc_i = fma(double(ri), double(ri), acc_i);
                acc_b = fma(bi, bi, acc_b);
            }
        }
    }
    rhs_cta_sum(acc_i, acc_b, a.part_init + int64_t(blockIdx.x) * 64, a.part_init + int64_t(blockIdx.x) * 64 + 32);
}

template <typename S>
__global__ void __launch_bounds__(kThreads, 3) k_rhs_row(RhsArgs a) {
    constexpr int V = RhsVec<S>::V, L = 32 / V;
    wait_prior_grid();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / L, ll = lane % L;
    const S *val = static_cast<const S *>(a.val);
    S *R = static_cast<S *>(a.R);
    const S *P = static_cast<const S *>(a.P);
    // phases: lane j (lane-per-column form) and the lane's V columns
    const bool mine = lane < a.k;
    const int32_t ph = mine ? *reinterpret_cast<const volatile int32_t *>(&a.st[lane].phase) : PH_DONE;
    const bool init = ph == PH_SETUP;
    const bool act = init || ph == PH_RUN;
    bool run[V], run_any = false, run_all = true;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int j = ll * V + v;
        run[v] = j < a.k && *reinterpret_cast<const volatile int32_t *>(&a.st[j].phase) == PH_RUN;
        run_any |= run[v];
        run_all &= run[v];
    }
    const bool any_init = __syncthreads_or(init) != 0;   // uniform over the CTA
    const bool any_run = __any_sync(0xffffffffu, run_any);
    RhsAcc<S> acc[V];
    // r = r - A p for the columns in PH_RUN: V matrix rows per warp
    for (int32_t ti = blockIdx.x; any_run && ti < a.n_rtiles; ti += gridDim.x) {
        const Tile t = a.rtiles[ti];
        // the row offsets of the next step are loaded one step ahead
        int32_t sn = t.begin + warp * V + sub < t.end ? a.row_ptr[t.begin + warp * V + sub] : 0;
        int32_t en = t.begin + warp * V + sub < t.end ? a.row_ptr[t.begin + warp * V + sub + 1] : 0;
        for (int32_t r0 = t.begin + warp * V; r0 < t.end; r0 += kWarps * V) {
            const int32_t row = r0 + sub;
            const bool valid = row < t.end;
            const int32_t s = sn, len = en - sn;
            const int32_t rn = row + kWarps * V;
            sn = rn < t.end ? a.row_ptr[rn] : 0;
            en = rn < t.end ? a.row_ptr[rn + 1] : 0;
            const int32_t len_max = __reduce_max_sync(0xffffffffu, len);
            const int64_t ix = int64_t(row) * kRhsStride + ll * V;
            S old[V], d[V];
            if (valid && run_any) RhsVec<S>::ld_rw(R + ix, old);
            rhs_vdot<S>(a.col_idx, val, s, len, len_max, P, ll * V, valid && run_any, d);
            if (valid && run_any) {
                S ri[V];
#pragma unroll
                for (int v = 0; v < V; ++v) ri[v] = old[v] - d[v];
                if (run_all) {
                    RhsVec<S>::st(R + ix, ri);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (run[v]) R[ix + v] = ri[v];
                }
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (run[v]) acc[v].add(ri[v], ri[v]);
            }
        }
    }
    double vr[V];
#pragma unroll
    for (int v = 0; v < V; ++v) vr[v] = acc[v].get();
    rhs_cta_sum_v<V>(vr, 0.0, a.part + int64_t(blockIdx.x) * 64);

    if (!rhs_arrive(&a.cnt[0], gridDim.x)) return;
    // rho of a restarting column (and ||b||^2) comes from k_rhs_row_init,
    // which ran just before with the same grid
    double rho, nb2 = 0.0;
    rhs_final_sums(any_init ? a.part_init : a.part, gridDim.x, 0, rho);
    double rho_run;
    rhs_final_sums(a.part, gridDim.x, 0, rho_run);
    if (any_init) rhs_final_sums(a.part_init, gridDim.x, 1, nb2);
    if (!init) rho = rho_run;
    if (threadIdx.x < 32 && mine && act) {
        SysState *st = a.st + lane;
        if (init) {
            st->nb = sqrt(nb2);
            st->rho0 = rho;
        }
        const double nb = st->nb;
        st->rho = rho;
        if (nb == 0.0) {
            st->relres_rec = 0.0;
            rhs_done(a, st, 0);
        } else {
            const double rel = sqrt(rho) / nb;
            st->relres_rec = rel;
            if (rel <= st->tol) {
                if (init || !st->stop_on_true) rhs_done(a, st, 0);
                else {
                    st->since = 0;
                    st->phase = PH_SETUP;
                }
            } else if (st->iters >= st->maxit) {
                rhs_done(a, st, 1);
            } else if (!init && st->inner_tol2 > 0.0 &&
                       (rho <= st->inner_tol2 * st->rho0 || rho > 4.0 * st->rho0)) {
                st->since = 0;
                st->phase = PH_SETUP;
            } else {
                st->phase = init ? PH_FIRST : PH_RUN;
            }
        }
    }
    if (threadIdx.x == 0) a.cnt[0] = 0;
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_rhs_col(RhsArgs a) {
    constexpr int V = RhsVec<S>::V, L = 32 / V;
    wait_prior_grid();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / L, ll = lane % L;
    const bool mine = lane < a.k;
    const int32_t ph = mine ? *reinterpret_cast<const volatile int32_t *>(&a.st[lane].phase) : PH_DONE;
    const bool act = ph == PH_FIRST || ph == PH_RUN;
    bool on[V], on_any = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int j = ll * V + v;
        const int32_t pj = j < a.k ? *reinterpret_cast<const volatile int32_t *>(&a.st[j].phase) : PH_DONE;
        on[v] = pj == PH_FIRST || pj == PH_RUN;
        on_any |= on[v];
    }
    const bool any_act = __any_sync(0xffffffffu, on_any);
    const S *val = static_cast<const S *>(a.cval);
    const S *R = static_cast<const S *>(a.R);
    S *U = static_cast<S *>(a.U);
    RhsAcc<S> accs[V];
    for (int32_t ti = blockIdx.x; any_act && ti < a.n_ctiles; ti += gridDim.x) {
        const Tile t = a.ctiles[ti];
        // the column offsets of the next step are loaded one step ahead
        int32_t sn = t.begin + warp * V + sub < t.end ? a.col_ptr[t.begin + warp * V + sub] : 0;
        int32_t en = t.begin + warp * V + sub < t.end ? a.col_ptr[t.begin + warp * V + sub + 1] : 0;
        for (int32_t c0 = t.begin + warp * V; c0 < t.end; c0 += kWarps * V) {
            const int32_t col = c0 + sub;
            const bool valid = col < t.end;
            const int32_t s = sn, len = en - sn;
            const int32_t cn = col + kWarps * V;
            sn = cn < t.end ? a.col_ptr[cn] : 0;
            en = cn < t.end ? a.col_ptr[cn + 1] : 0;
            const int32_t len_max = __reduce_max_sync(0xffffffffu, len);
            S y[V];
            rhs_vdot<S>(a.row_idx, val, s, len, len_max, R, ll * V, valid && on_any, y);
            if (valid && on_any) {
                S uj[V];
                if constexpr (std::is_same<S, float>::value) {
                    const float wj = a.wf ? a.wf[col] : 1.0f;
#pragma unroll
                    for (int v = 0; v < V; ++v) uj[v] = a.wf ? __fmul_rn(wj, y[v]) : y[v];
                } else {
                    const double wj = a.w ? a.w[col] : 1.0;
#pragma unroll
                    for (int v = 0; v < V; ++v) uj[v] = a.w ? wj * y[v] : y[v];
                }
                // U of an inactive column is recomputed before its next use
                RhsVec<S>::st(U + int64_t(col) * kRhsStride + ll * V, uj);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (on[v]) accs[v].add(y[v], uj[v]);
            }
        }
    }
    double vr[V];
#pragma unroll
    for (int v = 0; v < V; ++v) vr[v] = accs[v].get();
    rhs_cta_sum_v<V>(vr, 0.0, a.part + int64_t(blockIdx.x) * 64);
    if (!rhs_arrive(&a.cnt[1], gridDim.x)) return;
    double phi;
    rhs_final_sums(a.part, gridDim.x, 0, phi);
    if (threadIdx.x < 32 && mine && act) {
        SysState *st = a.st + lane;
        st->phi = phi;
        const double rho = st->rho;
        if (ph == PH_FIRST) {
            if (!(phi > 0.0) || !isfinite(phi)) rhs_done(a, st, -4);
            else {
                st->beta = 0.0;
                st->gamma = __ddiv_rn(rho, phi);
            }
        } else {
            const double theta = st->theta;
            const double sq = __dsqrt_rn(__dmul_rn(theta, phi));
            const double q = __ddiv_rn(sq, rho);
            const double dd = __dmul_rn(__dsub_rn(q, 1.0), __dadd_rn(q, 1.0));
            if (!(dd > 0.0) || !isfinite(dd)) {
                if (st->stop_on_true) {
                    st->since = 0;
                    st->phase = PH_SETUP;
                } else {
                    rhs_done(a, st, -4);
                }
            } else {
                const double beta = __ddiv_rn(1.0, dd);
                st->beta = beta;
                st->gamma = __dmul_rn(__ddiv_rn(theta, rho), beta);
            }
        }
    }
    if (threadIdx.x == 0) a.cnt[1] = 0;
}

// p = beta p + gamma u in the storage type (FP32: float beta, gamma as in
// the single-right-hand-side update), theta partials, x = x + p in double.
template <typename S>
__device__ __forceinline__ S rhs_pnew(bool first, S beta, S gamma, S p, S u);
template <>
__device__ __forceinline__ double rhs_pnew<double>(bool first, double beta, double gamma, double p, double u) {
    return first ? __dmul_rn(gamma, u) : __dadd_rn(__dmul_rn(beta, p), __dmul_rn(gamma, u));
}
template <>
__device__ __forceinline__ float rhs_pnew<float>(bool first, float bf, float gf, float p, float u) {
    return first ? gf * u : fmaf(bf, p, gf * u);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_rhs_update(RhsArgs a) {
    constexpr int V = RhsVec<S>::V, L = 32 / V;
    wait_prior_grid();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / L, ll = lane % L;
    const bool mine = lane < a.k;
    const int32_t ph = mine ? *reinterpret_cast<const volatile int32_t *>(&a.st[lane].phase) : PH_DONE;
    const bool act = ph == PH_FIRST || ph == PH_RUN;
    bool on[V], first[V], on_any = false, first_any = false;
    S beta[V], gamma[V];   // rounded to the storage type once (FP32: float)
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int j = ll * V + v;
        const int32_t pj = j < a.k ? *reinterpret_cast<const volatile int32_t *>(&a.st[j].phase) : PH_DONE;
        on[v] = pj == PH_FIRST || pj == PH_RUN;
        first[v] = pj == PH_FIRST;
        beta[v] = S(on[v] ? a.st[j].beta : 0.0);
        gamma[v] = S(on[v] ? a.st[j].gamma : 0.0);
        on_any |= on[v];
        first_any |= first[v];
    }
    // the first update after a (re)start is rare: keep its FP64 flush of dX
    // out of the common path (predicated-off FP64 instructions still occupy
    // the FP64 pipe)
    first_any = __syncthreads_or(first_any) != 0;
    S *P = static_cast<S *>(a.P);
    const S *U = static_cast<const S *>(a.U);
    RhsAcc<S> accs[V];
    for (int32_t ti = blockIdx.x; on_any && ti < a.n_vtiles; ti += gridDim.x) {
        const Tile t = a.vtiles[ti];
        for (int32_t j = t.begin + warp * V + sub; j < t.end; j += kWarps * V) {
            const int64_t ix = int64_t(j) * kRhsStride + ll * V;
            S uj[V], pj[V], pn[V];
            RhsVec<S>::ld_rw(U + ix, uj);
            RhsVec<S>::ld_rw(P + ix, pj);
#pragma unroll
            for (int v = 0; v < V; ++v) pn[v] = on[v] ? rhs_pnew<S>(first[v], beta[v], gamma[v], pj[v], uj[v]) : pj[v];
            RhsVec<S>::st(P + ix, pn);
            if constexpr (std::is_same<S, float>::value) {
                const float wi = a.winvf ? a.winvf[j] : 1.0f;
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (on[v]) accs[v].add(pn[v], a.winvf ? __fmul_rn(pn[v], wi) : pn[v]);
                // x accumulates in the float block dX during an inner solve;
                // the first update after a (re)start moves it into X
                float dx[V];
                RhsVec<float>::ld_rw(a.dX + ix, dx);
                if (first_any) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (first[v]) a.X[ix + v] = __dadd_rn(a.X[ix + v], double(dx[v]));
                }
#pragma unroll
                for (int v = 0; v < V; ++v) dx[v] = first[v] ? pn[v] : (on[v] ? __fadd_rn(dx[v], pn[v]) : dx[v]);
                RhsVec<float>::st(a.dX + ix, dx);
            } else {
                const double wi = a.winv ? a.winv[j] : 1.0;
                double xj[V];
                RhsVec<double>::ld_rw(a.X + ix, xj);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (on[v]) accs[v].add(pn[v], a.winv ? pn[v] * wi : pn[v]);
                    if (on[v]) xj[v] = __dadd_rn(xj[v], pn[v]);
                }
                RhsVec<double>::st(a.X + ix, xj);
            }
        }
    }
    double vr[V];
#pragma unroll
    for (int v = 0; v < V; ++v) vr[v] = accs[v].get();
    rhs_cta_sum_v<V>(vr, 0.0, a.part + int64_t(blockIdx.x) * 64);
    if (!rhs_arrive(&a.cnt[2], gridDim.x)) return;
    double theta;
    rhs_final_sums(a.part, gridDim.x, 0, theta);
    if (threadIdx.x < 32 && mine && act) {
        SysState *st = a.st + lane;
        st->theta = theta;
        const int64_t k = st->iters;
        if (st->hist && k < st->hist_cap) {
            double *h = st->hist + 5 * k;
            h[0] = st->rho;
            h[1] = st->phi;
            h[2] = st->beta;
            h[3] = st->gamma;
            h[4] = theta;
        }
        st->iters = k + 1;
        st->since += 1;
        if (st->refine > 0 && st->since >= st->refine) {
            st->since = 0;
            st->phase = PH_SETUP;
        } else {
            st->phase = PH_RUN;
        }
    }
    if (threadIdx.x == 0) a.cnt[2] = 0;
}

// FP32 storage, end of a solve: X = X + dX, dX = 0 (the updates of the last
// inner solve).
__global__ void __launch_bounds__(kThreads) k_rhs_flush(double *X, float *dX, int64_t count) {
    for (int64_t i = blockIdx.x * int64_t(kThreads) + threadIdx.x; i < count; i += int64_t(gridDim.x) * kThreads) {
        X[i] = __dadd_rn(X[i], double(dX[i]));
        dX[i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

void free_rhs(plss_ctx *c) {
    RhsState *r = c->rhs;
    if (!r) return;
    for (auto &kv : r->graphs) cudaGraphExecDestroy(kv.second);
    void *ptrs[] = {r->d_B, r->d_X, r->d_dX, r->d_R, r->d_P, r->d_U, r->d_part, r->d_st, r->d_cnt,
                    r->d_active, r->d_rt, r->d_ct, r->d_vt};
    for (void *p : ptrs) dfree(p);
    if (r->h_st) cudaFreeHost(r->h_st);
    if (r->h_active) cudaFreeHost(r->h_active);
    delete r;
    c->rhs = nullptr;
}

static void rhs_tiles(int64_t count, std::vector<Tile> &out) {
    if (count == 0) out.push_back({0, 0, 0, 32});
    for (int64_t i = 0; i < count; i += kRhsRowsPerTile)
        out.push_back({0, int32_t(i), int32_t(std::min<int64_t>(count, i + kRhsRowsPerTile)), 32});
}

static plss_status rhs_prepare(plss_ctx *c) {
    if (c->rhs) return PLSS_OK;
    RhsState *r = new RhsState();
    c->rhs = r;
    std::vector<Tile> rt, ct, vt;
    rhs_tiles(c->m, rt);
    rhs_tiles(c->n, ct);
    rhs_tiles(c->n, vt);
    r->n_rt = int32_t(rt.size());
    r->n_ct = int32_t(ct.size());
    r->n_vt = int32_t(vt.size());
    const size_t sb = c->f32 ? 4 : 8;
    const size_t maxt = size_t(std::max(1, c->nsm * kCtasPerSm));   // one partial per CTA
    plss_status st;
    auto up = [&](Tile **d, const std::vector<Tile> &h) -> plss_status {
        plss_status s2 = dalloc(reinterpret_cast<void **>(d), h.size() * sizeof(Tile), "rhs tiles");
        if (s2 != PLSS_OK) return s2;
        if (cudaMemcpy(*d, h.data(), h.size() * sizeof(Tile), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "tile upload failed");
        return PLSS_OK;
    };
    if ((st = dalloc(reinterpret_cast<void **>(&r->d_B), 8 * kRhsStride * size_t(c->m), "B")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&r->d_X), 8 * kRhsStride * size_t(c->n), "X")) != PLSS_OK ||
        (c->f32 && (st = dalloc(reinterpret_cast<void **>(&r->d_dX), 4 * kRhsStride * size_t(c->n), "dX")) != PLSS_OK) ||
        (st = dalloc(&r->d_R, sb * kRhsStride * size_t(c->m), "R")) != PLSS_OK ||
        (st = dalloc(&r->d_P, sb * kRhsStride * size_t(c->n), "P")) != PLSS_OK ||
        (st = dalloc(&r->d_U, sb * kRhsStride * size_t(c->n), "U")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&r->d_part), 2 * 8 * 64 * maxt, "partials")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&r->d_st), sizeof(SysState) * kRhsMax, "state")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&r->d_cnt), 16, "counters")) != PLSS_OK ||
        (st = dalloc(reinterpret_cast<void **>(&r->d_active), 16, "active")) != PLSS_OK ||
        (st = up(&r->d_rt, rt)) != PLSS_OK || (st = up(&r->d_ct, ct)) != PLSS_OK ||
        (st = up(&r->d_vt, vt)) != PLSS_OK) {
        free_rhs(c);
        return st;
    }
    if (cudaMemset(r->d_cnt, 0, 16) != cudaSuccess ||
        cudaMemset(r->d_P, 0, sb * kRhsStride * size_t(c->n)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&r->h_st), sizeof(SysState) * kRhsMax) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&r->h_active), 16) != cudaSuccess) {
        free_rhs(c);
        return fail(PLSS_ERR_CUDA, "set-up of the right-hand-side buffers failed");
    }
    return PLSS_OK;
}

static RhsArgs rhs_args(plss_ctx *c, int32_t k, bool w_on) {
    RhsState *r = c->rhs;
    RhsArgs a;
    a.row_ptr = c->d_row_ptr;
    a.col_idx = c->d_col_idx;
    a.val = c->d_val;
    a.col_ptr = c->d_col_ptr;
    a.row_idx = c->d_row_idx;
    a.cval = c->d_cval;
    a.rtiles = r->d_rt;
    a.ctiles = r->d_ct;
    a.vtiles = r->d_vt;
    a.n_rtiles = r->n_rt;
    a.n_ctiles = r->n_ct;
    a.n_vtiles = r->n_vt;
    a.k = k;
    a.m = c->m;
    a.n = c->n;
    a.st = r->d_st;
    a.part = r->d_part;
    a.part_init = r->d_part + 64 * std::max(1, c->nsm * kCtasPerSm);
    a.cnt = r->d_cnt;
    a.n_active = r->d_active;
    a.B = r->d_B;
    a.X = r->d_X;
    a.dX = r->d_dX;
    a.R = r->d_R;
    a.P = r->d_P;
    a.U = r->d_U;
    a.w = w_on ? c->d_w : nullptr;
    a.winv = w_on ? c->d_w + c->n : nullptr;
    a.wf = w_on && c->d_wf ? c->d_wf : nullptr;
    a.winvf = w_on && c->d_wf ? c->d_wf + c->n : nullptr;
    return a;
}

// Resident CTAs per SM of a kernel (at most kCtasPerSm: the partials hold
// one entry per CTA of nsm * kCtasPerSm).
template <typename K>
static int rhs_occupancy(K kernel) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    return std::min(n, kCtasPerSm);
}

static cudaError_t rhs_body(plss_ctx *c, const RhsArgs &a, cudaStream_t s) {
    // grids of one wave: every CTA resident at once
    const int orow = c->f32 ? rhs_occupancy(k_rhs_row<float>) : rhs_occupancy(k_rhs_row<double>);
    const int ocol = c->f32 ? rhs_occupancy(k_rhs_col<float>) : rhs_occupancy(k_rhs_col<double>);
    const int oupd = c->f32 ? rhs_occupancy(k_rhs_update<float>) : rhs_occupancy(k_rhs_update<double>);
    const int gr = std::max(1, std::min(a.n_rtiles, c->nsm * orow));
    const int gc = std::max(1, std::min(a.n_ctiles, c->nsm * ocol));
    const int gv = std::max(1, std::min(a.n_vtiles, c->nsm * oupd));
    cudaError_t e;
    if (c->f32) {
        if ((e = launch_pdl(k_rhs_col<float>, gc, s, a)) != cudaSuccess) return e;
        if ((e = launch_pdl(k_rhs_update<float>, gv, s, a)) != cudaSuccess) return e;
        if ((e = launch_pdl(k_rhs_row_init<float>, gr, s, a)) != cudaSuccess) return e;
        e = launch_pdl(k_rhs_row<float>, gr, s, a);
    } else {
        if ((e = launch_pdl(k_rhs_col<double>, gc, s, a)) != cudaSuccess) return e;
        if ((e = launch_pdl(k_rhs_update<double>, gv, s, a)) != cudaSuccess) return e;
        if ((e = launch_pdl(k_rhs_row_init<double>, gr, s, a)) != cudaSuccess) return e;
        e = launch_pdl(k_rhs_row<double>, gr, s, a);
    }
    return e;
}

static plss_status rhs_graph(plss_ctx *c, int chunk, int32_t k, bool w_on, cudaGraphExec_t *out) {
    RhsState *r = c->rhs;
    const int key = (chunk * 64 + k) * 2 + (w_on ? 1 : 0);
    auto it = r->graphs.find(key);
    if (it != r->graphs.end()) {
        *out = it->second;
        return PLSS_OK;
    }
    const RhsArgs a = rhs_args(c, k, w_on);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "begin capture failed");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < chunk && e == cudaSuccess; ++i) e = rhs_body(c, a, c->cap_stream);
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(PLSS_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return fail(PLSS_ERR_CUDA, "instantiate failed: %s", cudaGetErrorString(e3));
    r->graphs[key] = ge;
    *out = ge;
    return PLSS_OK;
}

// Moves a row-major (rows x k) block between the caller and a stride-32 block.
static plss_status rhs_put(double *dst, const double *src, int64_t rows, int32_t k, bool dev, cudaStream_t s) {
    if (rows == 0) return PLSS_OK;
    if (!src) {
        if (cudaMemsetAsync(dst, 0, 8 * kRhsStride * size_t(rows), s) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "memset failed");
        return PLSS_OK;
    }
    if (cudaMemsetAsync(dst, 0, 8 * kRhsStride * size_t(rows), s) != cudaSuccess ||
        cudaMemcpy2DAsync(dst, 8 * kRhsStride, src, 8 * size_t(k), 8 * size_t(k), size_t(rows),
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "copy of a right-hand-side block failed");
    return PLSS_OK;
}

plss_status run_rhs(plss_ctx *c, int32_t k, const double *B, const double *X0, double *X,
                    const plss_opts *o, plss_result *res) {
    TraceRange tr("plss: solve (many right-hand sides)");
    plss_status st = check_opts(o);
    if (st != PLSS_OK) return st;
    if (c->nsys != 1) return fail(PLSS_ERR_INVALID, "plss_solve_rhs needs a single-system context");
    if (k < 1 || k > kRhsMax) return fail(PLSS_ERR_INVALID, "nrhs must be in [1, %d]", kRhsMax);
    if (o->sketch != PLSS_SKETCH_RESIDUAL) return fail(PLSS_ERR_INVALID, "plss_solve_rhs runs the residual sketch");
    c->state_valid = false;   // x and b of the context are overwritten: nothing to resume
    if (o->refine_mode != PLSS_REFINE_RESTART)
        return fail(PLSS_ERR_INVALID, "plss_solve_rhs refines by restarts only (refine_mode RESTART)");
    if ((c->m > 0 && !B) || (c->n > 0 && !X)) return fail(PLSS_ERR_INVALID, "NULL block");
    if ((st = rhs_prepare(c)) != PLSS_OK) return st;
    RhsState *r = c->rhs;
    cudaStream_t s = static_cast<cudaStream_t>(o->stream);
    const bool dev = o->io_device != 0;
    if ((st = rhs_put(r->d_B, B, c->m, k, dev, s)) != PLSS_OK) return st;
    if ((st = rhs_put(r->d_X, X0, c->n, k, dev, s)) != PLSS_OK) return st;
    if (r->d_dX && c->n > 0 && cudaMemsetAsync(r->d_dX, 0, 4 * kRhsStride * size_t(c->n), s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "memset failed");
    if ((st = ensure_weights(c, o->w_mode, s)) != PLSS_OK) return st;
    const bool w_on = o->w_mode != PLSS_W_IDENTITY;
    if (o->hist_cap > 0 && o->hist_cap > c->hist_cap_alloc) {
        dfree(c->d_hist);
        c->d_hist = nullptr;
        c->hist_cap_alloc = 0;
        if ((st = dalloc(reinterpret_cast<void **>(&c->d_hist), size_t(o->hist_cap) * 40, "hist")) != PLSS_OK) return st;
        c->hist_cap_alloc = o->hist_cap;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PLSS_ERR_CUDA, "synchronize failed");
    const int64_t maxit = o->maxit < 0 ? c->n : o->maxit;
    for (int32_t j = 0; j < kRhsMax; ++j) {
        SysState z;
        std::memset(&z, 0, sizeof z);
        z.tol = o->tol;
        z.maxit = maxit;
        z.refine = c->f32 ? std::max<int64_t>(0, o->refine_period) : 0;
        z.inner_tol2 = c->f32 ? o->inner_tol * o->inner_tol : 0.0;
        z.stop_on_true = (c->f32 || o->stop_on_true) ? 1 : 0;
        z.phase = j < k ? PH_SETUP : PH_DONE;
        if (j == 0 && o->hist_cap > 0) {
            z.hist = c->d_hist;
            z.hist_cap = o->hist_cap;
        }
        r->h_st[j] = z;
    }
    *r->h_active = k;
    if (cudaMemcpyAsync(r->d_st, r->h_st, sizeof(SysState) * kRhsMax, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(r->d_active, r->h_active, 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(c->ev0, s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "state upload failed");
    const int64_t body_cap = 2 * (maxit + 2) + 8;
    int64_t bodies = 0;
    int chunk = 1;
    for (;;) {
        cudaGraphExec_t g;
        if ((st = rhs_graph(c, chunk, k, w_on, &g)) != PLSS_OK) return st;
        if (cudaGraphLaunch(g, s) != cudaSuccess ||
            cudaMemcpyAsync(r->h_active, r->d_active, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "iteration launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        bodies += chunk;
        if (*r->h_active <= 0) break;
        if (bodies > body_cap) return fail(PLSS_ERR_TIMEOUT, "iteration driver exceeded %lld bodies", (long long)body_cap);
        chunk = std::min(chunk * 4, kMaxChunk);
    }
    if (r->d_dX && c->n > 0) {
        const int64_t cnt = int64_t(kRhsStride) * c->n;
        const int grid = int(std::min<int64_t>((cnt + kThreads - 1) / kThreads, int64_t(c->nsm) * kCtasPerSm));
        k_rhs_flush<<<grid, kThreads, 0, s>>>(r->d_X, r->d_dX, cnt);
    }
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(c->ev1, s) != cudaSuccess ||
        cudaMemcpyAsync(r->h_st, r->d_st, sizeof(SysState) * kRhsMax, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpy2DAsync(X, 8 * size_t(k), r->d_X, 8 * kRhsStride, 8 * size_t(k), size_t(c->n),
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "reading results failed");
    if (o->hist_cap > 0) {
        const int64_t kk = std::min<int64_t>(o->hist_cap, r->h_st[0].iters);
        if (kk > 0 && cudaMemcpy(o->hist, c->d_hist, size_t(kk) * 40, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "reading the history failed");
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    // true residuals, one column at a time through the context's vectors
    std::vector<double> col(static_cast<size_t>(std::max<int64_t>(c->m, c->n)));
    plss_status overall = PLSS_OK;
    for (int32_t j = 0; j < k; ++j) {
        // x_j and b_j into the single-vector buffers (strided device copies)
        if (cudaMemcpy2DAsync(c->d_x, 8, r->d_X + j, 8 * kRhsStride, 8, size_t(c->n), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpy2DAsync(c->d_b, 8, r->d_B + j, 8 * kRhsStride, 8, size_t(c->m), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(PLSS_ERR_CUDA, "column copy failed");
        c->h_st[0].nb = r->h_st[j].nb;
        std::vector<double> rel;
        if ((st = true_relres(c, s, rel)) != PLSS_OK) return st;
        const SysState &z = r->h_st[j];
        if (res) {
            res[j].status = z.status;
            res[j].reserved = 0;
            res[j].iters = z.iters;
            res[j].relres_rec = z.relres_rec;
            res[j].relres_true = rel[0];
            res[j].seconds = double(ms) * 1e-3;
        }
        if (overall == PLSS_OK && z.status != PLSS_OK) overall = plss_status(z.status);
    }
    return overall;
}

}  // namespace plss

using namespace plss;

extern "C" plss_status plss_solve_rhs(plss_ctx *ctx, int32_t nrhs, const double *B, const double *X0,
                                      double *X, const plss_opts *o, plss_result *res) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    return run_rhs(ctx, nrhs, B, X0, X, o, res);
}
