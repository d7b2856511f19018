// plss_kernels.cu -- residual-sketch PLSS sweeps for sm_103a.
//
// One iteration of Algorithm 1 (Sec. 5) for every active system of a packed
// context is the body  [column sweep] -> [update] -> [row sweep]:
//
//   column sweep  y = A^T r, u = W y, phi = y^T u; the last tile of a system
//                 then takes the scalar step of Theorem 4.1:
//                 s = sqrt(theta phi), beta = 1/((s/rho - 1)(s/rho + 1)),
//                 gamma = (theta/rho) beta   (or beta = 0, gamma = rho/phi on
//                 the first update after a (re)start, Algorithm 1's
//                 initialisation p = (rho/phi) W y)
//   update        p = beta p + gamma u, theta = p^T W^{-1} p, x = x + p
//   row sweep     r = r - A p, rho = r^T r (or r = b - A x in double after a
//                 (re)start); the last tile then applies the stopping rule
//                 sqrt(rho)/||b|| <= tol (Sec. 5) and the maxit cap.
//
// The sweeps are HBM-bandwidth bound (about 2 flops per 12-16 bytes), so the
// kernels are plain CUDA-core code built for memory-level parallelism:
//   * a tile is a run of whole rows (columns) holding at most 2,048
//     nonzeros; its nonzeros are streamed with coalesced loads, 8 per thread
//     issued back to back with their gathers, and the products are staged
//     in shared memory;
//   * the segments are then summed out of shared memory by groups of G
//     lanes (G picked per tile from its mean segment length) with a
//     warp-shuffle tree; a segment longer than a tile gets a tile of its own
//     that the whole CTA streams;
//   * each CTA owns a contiguous range of tiles; per-tile FP64 partial sums
//     of rho / phi / theta are written to global memory and each CTA
//     announces its tiles with one atomic per system it touched; the CTA
//     that completes a system sums that system's partials in tile order
//     (deterministic for a given schedule) and takes its scalar step.
#include <cuda_runtime.h>

#include "plss_dev.cuh"
#include "plss_launch.h"

namespace plss {

constexpr int kUnroll = 8;                       // nonzeros per thread per tile
constexpr int kStreamNnz = kThreads * kUnroll;   // nonzeros staged per tile

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// Fixed-order sum over the CTA of N doubles. Every thread calls it; the
// result is valid in thread 0.
template <int N>
__device__ __forceinline__ void cta_sum(double (&v)[N]) {
    __shared__ double sh[N][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) sh[i][warp] = v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < kWarps; ++k) s += sh[i][k];
            v[i] = s;
        }
    }
}

// Products val[z0+k] * x[idx[z0+k]] for k < nz (nz <= kStreamNnz) into
// prod[k]: every thread issues its 8 index/value loads, then its 8 gathers,
// before using any of them.
template <typename VT, typename XT, typename PT>
__device__ __forceinline__ void stage_products(const int32_t *__restrict__ idx,
                                               const VT *__restrict__ val, int32_t z0, int32_t nz,
                                               const XT *__restrict__ x, PT *prod) {
    int32_t c[kUnroll];
    VT v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int32_t k = threadIdx.x + u * kThreads;
        const bool in = k < nz;
        c[u] = in ? __ldg(idx + z0 + k) : 0;
        v[u] = in ? __ldg(val + z0 + k) : VT(0);
    }
    XT g[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int32_t k = threadIdx.x + u * kThreads;
        g[u] = k < nz ? __ldg(x + c[u]) : XT(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int32_t k = threadIdx.x + u * kThreads;
        if (k < nz) prod[k] = PT(v[u]) * PT(g[u]);
    }
}

// Dot product of one long segment [s, e) with a dense vector, streamed by
// the whole CTA with 8 independent accumulators per thread; lane partials
// combined in a fixed order in double (result in thread 0).
template <typename VT, typename XT, typename ACC>
__device__ __forceinline__ double cta_dot(const int32_t *__restrict__ idx,
                                          const VT *__restrict__ val, int32_t s, int32_t e,
                                          const XT *__restrict__ x) {
    ACC acc[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) acc[u] = ACC(0);
    for (int32_t base = s; base < e; base += kStreamNnz) {
        int32_t c[kUnroll];
        VT v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t k = base + threadIdx.x + u * kThreads;
            const bool in = k < e;
            c[u] = in ? __ldg(idx + k) : 0;
            v[u] = in ? __ldg(val + k) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int32_t k = base + threadIdx.x + u * kThreads;
            if (k < e) acc[u] = fma_t(ACC(v[u]), ACC(__ldg(x + c[u])), acc[u]);
        }
    }
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) t += double(acc[u]);
    double v1[1] = {t};
    cta_sum<1>(v1);
    return v1[0];
}

// Calls body(seg, s, e, gl, valid) for each segment of the tile with groups
// of G lanes; the loop is warp-uniform.
template <int G, typename F>
__device__ __forceinline__ void for_segments(const int32_t *__restrict__ ptr, const Tile &t, F &&body) {
    constexpr int SPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane & (G - 1);
    for (int32_t base = t.begin + warp * SPW; base < t.end; base += kWarps * SPW) {
        const int32_t seg = base + gid;
        const bool valid = seg < t.end;
        const int32_t s = valid ? __ldg(ptr + seg) : 0;
        const int32_t e = valid ? __ldg(ptr + seg + 1) : 0;
        body(seg, s, e, gl, valid);
    }
}

// Sum of the staged products of one segment over the G lanes of a group
// (lane-strided, then a shuffle tree); valid in every lane of the group.
template <int G, typename PT>
__device__ __forceinline__ PT group_sum(const PT *prod, int32_t s, int32_t e, int gl) {
    PT acc = PT(0);
    for (int32_t k = s + gl; k < e; k += G) acc += prod[k];
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Contiguous, balanced share of n tiles for this CTA.
__device__ __forceinline__ void tile_range(int32_t n, int32_t &t0, int32_t &t1) {
    const int32_t per = n / int32_t(gridDim.x), rem = n % int32_t(gridDim.x);
    const int32_t b = int32_t(blockIdx.x);
    t0 = b * per + (b < rem ? b : rem);
    t1 = t0 + per + (b < rem ? 1 : 0);
}

// This CTA has finished `pending` tiles of a system with `total` tiles:
// returns (to all threads) whether that completed the system.
__device__ __forceinline__ bool arrive(uint32_t *cnt, uint32_t pending, int32_t total) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(cnt, pending);
        s_last = prev + pending == uint32_t(total);
    }
    __syncthreads();
    const bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ int32_t load_phase(const SysState *st) {
    return *reinterpret_cast<const volatile int32_t *>(&st->phase);
}

__device__ __forceinline__ void finish_system(const SweepArgs &a, SysState *st, int32_t status) {
    st->status = status;
    st->phase = PH_DONE;
    atomicSub(a.n_active, 1);
}

// ---------------------------------------------------------------------------
// Row sweep: r = r - A p (or r = b - A x), rho = r^T r
// ---------------------------------------------------------------------------

template <int G, typename S>
__device__ __forceinline__ void row_tile(const SweepArgs &a, const Tile &t, bool init,
                                         double &acc_r, double &acc_b, double *smem) {
    const S *__restrict__ val = static_cast<const S *>(a.val);
    S *__restrict__ r = static_cast<S *>(a.r);
    const int32_t z0 = __ldg(a.row_ptr + t.begin);
    const int32_t nz = __ldg(a.row_ptr + t.end) - z0;
    if (init) {
        stage_products<S, double, double>(a.col_idx, val, z0, nz, a.x, smem);
        __syncthreads();
        const double *prod = smem - z0;
        for_segments<G>(a.row_ptr, t, [&](int32_t row, int32_t s, int32_t e, int gl, bool valid) {
            const double d = group_sum<G>(prod, s, e, gl);
            if (valid && gl == 0) {
                const double bi = a.b[row];
                const S ri = S(bi - d);
                r[row] = ri;
                acc_r += double(ri) * double(ri);
                acc_b += bi * bi;
            }
        });
    } else {
        S *sp = reinterpret_cast<S *>(smem);
        stage_products<S, S, S>(a.col_idx, val, z0, nz, static_cast<const S *>(a.p), sp);
        __syncthreads();
        const S *prod = sp - z0;
        for_segments<G>(a.row_ptr, t, [&](int32_t row, int32_t s, int32_t e, int gl, bool valid) {
            const S d = group_sum<G>(prod, s, e, gl);
            if (valid && gl == 0) {
                const S ri = r[row] - d;
                r[row] = ri;
                acc_r += double(ri) * double(ri);
            }
        });
    }
    __syncthreads();
}

template <typename S>
__device__ __forceinline__ void row_tile_cta(const SweepArgs &a, const Tile &t, bool init,
                                             double &acc_r, double &acc_b) {
    const S *__restrict__ val = static_cast<const S *>(a.val);
    S *__restrict__ r = static_cast<S *>(a.r);
    const int32_t row = t.begin;
    const int32_t s = a.row_ptr[row], e = a.row_ptr[row + 1];
    double d;
    if (init) d = cta_dot<S, double, double>(a.col_idx, val, s, e, a.x);
    else d = cta_dot<S, S, S>(a.col_idx, val, s, e, static_cast<const S *>(a.p));
    if (threadIdx.x == 0) {
        if (init) {
            const double bi = a.b[row];
            const S ri = S(bi - d);
            r[row] = ri;
            acc_r += double(ri) * double(ri);
            acc_b += bi * bi;
        } else {
            const S ri = r[row] - S(d);
            r[row] = ri;
            acc_r += double(ri) * double(ri);
        }
    }
}

__device__ void finish_row(const SweepArgs &a, int32_t sys, bool init) {
    const SysDesc d = a.desc[sys];
    double v[2] = {0.0, 0.0};
    for (int32_t i = threadIdx.x; i < d.rt_count; i += kThreads) {
        v[0] += __ldcg(a.part_row + 2 * (d.rt_begin + i));
        v[1] += __ldcg(a.part_row + 2 * (d.rt_begin + i) + 1);
    }
    cta_sum<2>(v);
    if (threadIdx.x != 0) return;
    SysState *st = a.st + sys;
    st->cnt_row = 0;
    const double rho = v[0];
    if (init) {
        st->nb = sqrt(v[1]);
        st->rho0 = rho;
    }
    const double nb = st->nb;
    st->rho = rho;
    if (nb == 0.0) {
        st->relres_rec = 0.0;
        finish_system(a, st, 0);
        return;
    }
    const double rel = sqrt(rho) / nb;
    st->relres_rec = rel;
    if (rel <= st->tol) {
        if (init || !st->stop_on_true) {
            finish_system(a, st, 0);
        } else {
            st->since = 0;
            st->phase = PH_SETUP;   // confirm on b - A x before stopping
        }
    } else if (st->iters >= st->maxit) {
        finish_system(a, st, 1);
    } else if (!init && st->inner_tol2 > 0.0 && rho <= st->inner_tol2 * st->rho0) {
        st->since = 0;
        st->phase = PH_SETUP;       // inner solve done: refine from b - A x
    } else {
        st->phase = init ? PH_FIRST : PH_RUN;
    }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_row_sweep(SweepArgs a) {
    __shared__ __align__(16) double smem[kStreamNnz];
    int32_t t0, t1;
    tile_range(a.n_rtiles, t0, t1);
    int32_t cur = -1;
    uint32_t pending = 0;
    bool active = false, init = false;
    for (int32_t ti = t0; ti < t1; ++ti) {
        const Tile t = a.rtiles[ti];
        if (t.sys != cur) {
            if (pending && arrive(&a.st[cur].cnt_row, pending, a.desc[cur].rt_count))
                finish_row(a, cur, init);
            cur = t.sys;
            pending = 0;
            const int32_t ph = load_phase(a.st + cur);
            active = ph == PH_SETUP || ph == PH_RUN;
            init = ph == PH_SETUP;
        }
        if (!active) continue;
        double acc[2] = {0.0, 0.0};
        switch (t.group) {
            case 0: row_tile_cta<S>(a, t, init, acc[0], acc[1]); break;
            case 1: row_tile<1, S>(a, t, init, acc[0], acc[1], smem); break;
            case 2: row_tile<2, S>(a, t, init, acc[0], acc[1], smem); break;
            case 4: row_tile<4, S>(a, t, init, acc[0], acc[1], smem); break;
            case 8: row_tile<8, S>(a, t, init, acc[0], acc[1], smem); break;
            case 16: row_tile<16, S>(a, t, init, acc[0], acc[1], smem); break;
            default: row_tile<32, S>(a, t, init, acc[0], acc[1], smem); break;
        }
        cta_sum<2>(acc);
        if (threadIdx.x == 0) {
            a.part_row[2 * ti] = acc[0];
            a.part_row[2 * ti + 1] = acc[1];
        }
        ++pending;
    }
    if (pending && arrive(&a.st[cur].cnt_row, pending, a.desc[cur].rt_count)) finish_row(a, cur, init);
}

// ---------------------------------------------------------------------------
// Column sweep: y = A^T r, u = W y, phi = y^T u, then the scalar step
// ---------------------------------------------------------------------------

template <typename S>
__device__ __forceinline__ void col_out(const SweepArgs &a, int32_t col, double y, double &acc) {
    const S uj = a.w ? S(a.w[col] * y) : S(y);
    static_cast<S *>(a.u)[col] = uj;
    acc += y * double(uj);
}

template <int G, typename S>
__device__ __forceinline__ void col_tile(const SweepArgs &a, const Tile &t, double &acc, double *smem) {
    const S *__restrict__ val = static_cast<const S *>(a.cval);
    const int32_t z0 = __ldg(a.col_ptr + t.begin);
    const int32_t nz = __ldg(a.col_ptr + t.end) - z0;
    S *sp = reinterpret_cast<S *>(smem);
    stage_products<S, S, S>(a.row_idx, val, z0, nz, static_cast<const S *>(a.r), sp);
    __syncthreads();
    const S *prod = sp - z0;
    for_segments<G>(a.col_ptr, t, [&](int32_t col, int32_t s, int32_t e, int gl, bool valid) {
        const S d = group_sum<G>(prod, s, e, gl);
        if (valid && gl == 0) col_out<S>(a, col, double(d), acc);
    });
    __syncthreads();
}

template <typename S>
__device__ __forceinline__ void col_tile_cta(const SweepArgs &a, const Tile &t, double &acc) {
    const int32_t col = t.begin;
    const int32_t s = a.col_ptr[col], e = a.col_ptr[col + 1];
    const double d = cta_dot<S, S, S>(a.row_idx, static_cast<const S *>(a.cval), s, e,
                                      static_cast<const S *>(a.r));
    if (threadIdx.x == 0) col_out<S>(a, col, double(S(d)), acc);
}

__device__ void finish_col(const SweepArgs &a, int32_t sys) {
    const SysDesc d = a.desc[sys];
    double v[1] = {0.0};
    for (int32_t i = threadIdx.x; i < d.ct_count; i += kThreads)
        v[0] += __ldcg(a.part_col + d.ct_begin + i);
    cta_sum<1>(v);
    if (threadIdx.x != 0) return;
    SysState *st = a.st + sys;
    st->cnt_col = 0;
    const double phi = v[0];
    st->phi = phi;
    const double rho = st->rho;
    if (st->phase == PH_FIRST) {
        // Algorithm 1 initialisation: p = (rho/phi) W y
        if (!(phi > 0.0) || !isfinite(phi)) { finish_system(a, st, -4); return; }
        st->beta = 0.0;
        st->gamma = __ddiv_rn(rho, phi);
    } else {
        // Theorem 4.1 as written in Algorithm 1
        const double theta = st->theta;
        const double s = __dsqrt_rn(__dmul_rn(theta, phi));
        const double q = __ddiv_rn(s, rho);
        const double dd = __dmul_rn(__dsub_rn(q, 1.0), __dadd_rn(q, 1.0));
        if (!(dd > 0.0) || !isfinite(dd)) {
            if (st->stop_on_true) {
                // the recursion lost orthogonality to rounding: restart from
                // b - A x (the next row sweep) instead of stopping
                st->since = 0;
                st->phase = PH_SETUP;
            } else {
                finish_system(a, st, -4);
            }
            return;
        }
        const double beta = __ddiv_rn(1.0, dd);
        st->beta = beta;
        st->gamma = __dmul_rn(__ddiv_rn(theta, rho), beta);
    }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_col_sweep(SweepArgs a) {
    __shared__ __align__(16) double smem[kStreamNnz];
    int32_t t0, t1;
    tile_range(a.n_ctiles, t0, t1);
    int32_t cur = -1;
    uint32_t pending = 0;
    bool active = false;
    for (int32_t ti = t0; ti < t1; ++ti) {
        const Tile t = a.ctiles[ti];
        if (t.sys != cur) {
            if (pending && arrive(&a.st[cur].cnt_col, pending, a.desc[cur].ct_count)) finish_col(a, cur);
            cur = t.sys;
            pending = 0;
            const int32_t ph = load_phase(a.st + cur);
            active = ph == PH_FIRST || ph == PH_RUN;
        }
        if (!active) continue;
        double acc[1] = {0.0};
        switch (t.group) {
            case 0: col_tile_cta<S>(a, t, acc[0]); break;
            case 1: col_tile<1, S>(a, t, acc[0], smem); break;
            case 2: col_tile<2, S>(a, t, acc[0], smem); break;
            case 4: col_tile<4, S>(a, t, acc[0], smem); break;
            case 8: col_tile<8, S>(a, t, acc[0], smem); break;
            case 16: col_tile<16, S>(a, t, acc[0], smem); break;
            default: col_tile<32, S>(a, t, acc[0], smem); break;
        }
        cta_sum<1>(acc);
        if (threadIdx.x == 0) a.part_col[ti] = acc[0];
        ++pending;
    }
    if (pending && arrive(&a.st[cur].cnt_col, pending, a.desc[cur].ct_count)) finish_col(a, cur);
}

// ---------------------------------------------------------------------------
// Update: p = beta p + gamma u, theta = p^T W^{-1} p, x = x + p
// ---------------------------------------------------------------------------

__device__ void finish_upd(const SweepArgs &a, int32_t sys) {
    const SysDesc d = a.desc[sys];
    double v[1] = {0.0};
    for (int32_t i = threadIdx.x; i < d.vt_count; i += kThreads)
        v[0] += __ldcg(a.part_upd + d.vt_begin + i);
    cta_sum<1>(v);
    if (threadIdx.x != 0) return;
    SysState *st = a.st + sys;
    st->cnt_upd = 0;
    const double theta = v[0];
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
        st->phase = PH_SETUP;   // periodic refinement: restart from b - A x
    } else {
        st->phase = PH_RUN;
    }
}

template <typename S>
__device__ __forceinline__ double update_tile(const SweepArgs &a, const Tile &t, bool first,
                                              double beta, double gamma) {
    S *__restrict__ p = static_cast<S *>(a.p);
    const S *__restrict__ u = static_cast<const S *>(a.u);
    double *__restrict__ x = a.x;
    const double *__restrict__ w = a.w;
    double acc = 0.0;
    constexpr int U = 4;
    for (int32_t base = t.begin; base < t.end; base += kThreads * U) {
        double uj[U], pj[U], xj[U], wj[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int32_t j = base + threadIdx.x + q * kThreads;
            const bool in = j < t.end;
            uj[q] = in ? double(u[j]) : 0.0;
            pj[q] = in && !first ? double(p[j]) : 0.0;
            xj[q] = in ? x[j] : 0.0;
            wj[q] = in && w ? w[j] : 1.0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int32_t j = base + threadIdx.x + q * kThreads;
            if (j < t.end) {
                const double pn = first ? __dmul_rn(gamma, uj[q])
                                        : __dadd_rn(__dmul_rn(beta, pj[q]), __dmul_rn(gamma, uj[q]));
                const S ps = S(pn);
                p[j] = ps;
                const double pd = double(ps);
                acc += w ? __ddiv_rn(__dmul_rn(pd, pd), wj[q]) : __dmul_rn(pd, pd);
                x[j] = __dadd_rn(xj[q], pd);
            }
        }
    }
    return acc;
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_update(SweepArgs a) {
    int32_t t0, t1;
    tile_range(a.n_vtiles, t0, t1);
    int32_t cur = -1;
    uint32_t pending = 0;
    bool active = false, first = false;
    double beta = 0.0, gamma = 0.0;
    for (int32_t ti = t0; ti < t1; ++ti) {
        const Tile t = a.vtiles[ti];
        if (t.sys != cur) {
            if (pending && arrive(&a.st[cur].cnt_upd, pending, a.desc[cur].vt_count)) finish_upd(a, cur);
            cur = t.sys;
            pending = 0;
            const int32_t ph = load_phase(a.st + cur);
            active = ph == PH_FIRST || ph == PH_RUN;
            first = ph == PH_FIRST;
            beta = a.st[cur].beta;
            gamma = a.st[cur].gamma;
        }
        if (!active) continue;
        double acc[1] = {update_tile<S>(a, t, first, beta, gamma)};
        cta_sum<1>(acc);
        if (threadIdx.x == 0) a.part_upd[ti] = acc[0];
        ++pending;
    }
    if (pending && arrive(&a.st[cur].cnt_upd, pending, a.desc[cur].vt_count)) finish_upd(a, cur);
}

// ---------------------------------------------------------------------------
// Auxiliary kernels: products in double, residual norms, column weights
// ---------------------------------------------------------------------------

template <int G>
__device__ __forceinline__ void spmv_segments(const int32_t *ptr, const Tile &t, const double *prod,
                                              double *out) {
    for_segments<G>(ptr, t, [&](int32_t seg, int32_t s, int32_t e, int gl, bool valid) {
        const double d = group_sum<G>(prod, s, e, gl);
        if (valid && gl == 0) out[seg] = d;
    });
}

// out[seg] = sum over the segment of val * v[idx] (double); with b given,
// part[tile] = sum over the tile of (b - out)^2 (residual norms).
template <typename S>
__global__ void __launch_bounds__(kThreads)
k_spmv(const int32_t *ptr, const int32_t *idx, const void *val_, const Tile *tiles, int32_t ntiles,
       const double *v, double *out, const double *b, double *part) {
    __shared__ __align__(16) double smem[kStreamNnz];
    const S *val = static_cast<const S *>(val_);
    for (int32_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tiles[ti];
        if (t.group == 0) {
            const int32_t s = ptr[t.begin], e = ptr[t.begin + 1];
            const double d = cta_dot<S, double, double>(idx, val, s, e, v);
            if (threadIdx.x == 0) out[t.begin] = d;
        } else {
            const int32_t z0 = ptr[t.begin];
            stage_products<S, double, double>(idx, val, z0, ptr[t.end] - z0, v, smem);
            __syncthreads();
            const double *prod = smem - z0;
            switch (t.group) {
                case 1: spmv_segments<1>(ptr, t, prod, out); break;
                case 2: spmv_segments<2>(ptr, t, prod, out); break;
                case 4: spmv_segments<4>(ptr, t, prod, out); break;
                case 8: spmv_segments<8>(ptr, t, prod, out); break;
                case 16: spmv_segments<16>(ptr, t, prod, out); break;
                default: spmv_segments<32>(ptr, t, prod, out); break;
            }
        }
        __syncthreads();
        if (b != nullptr) {
            double acc[1] = {0.0};
            for (int32_t i = t.begin + threadIdx.x; i < t.end; i += kThreads) {
                const double ri = b[i] - out[i];
                acc[0] += ri * ri;
            }
            cta_sum<1>(acc);
            if (threadIdx.x == 0) part[ti] = acc[0];
        }
        __syncthreads();
    }
}

// w_j from the squared norm of column j (segments of the CSC, ascending
// rows): mode 1 -> 1/||A_j||, mode 2 -> 1/||A_j||^2, empty column -> 1.
template <typename S>
__global__ void k_colweights(const int32_t *ptr, const void *val_, int64_t n, int32_t mode, double *w) {
    const S *val = static_cast<const S *>(val_);
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n;
         j += int64_t(gridDim.x) * blockDim.x) {
        double ss = 0.0;
        for (int32_t k = ptr[j]; k < ptr[j + 1]; ++k) {
            const double v = double(val[k]);
            ss = __dadd_rn(ss, __dmul_rn(v, v));
        }
        w[j] = ss == 0.0 ? 1.0 : (mode == 2 ? __ddiv_rn(1.0, ss) : __ddiv_rn(1.0, __dsqrt_rn(ss)));
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

static_assert(kStreamNnz == 2048, "tile nonzero capacity must match the host tile builder");

cudaError_t launch_row_sweep(const SweepArgs &a, bool f32, int grid, cudaStream_t s) {
    if (f32) k_row_sweep<float><<<grid, kThreads, 0, s>>>(a);
    else k_row_sweep<double><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_col_sweep(const SweepArgs &a, bool f32, int grid, cudaStream_t s) {
    if (f32) k_col_sweep<float><<<grid, kThreads, 0, s>>>(a);
    else k_col_sweep<double><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_update(const SweepArgs &a, bool f32, int grid, cudaStream_t s) {
    if (f32) k_update<float><<<grid, kThreads, 0, s>>>(a);
    else k_update<double><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_spmv(const int32_t *ptr, const int32_t *idx, const void *val, bool f32,
                        const Tile *tiles, int32_t ntiles, const double *v, double *out,
                        const double *b, double *part, int grid, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    if (f32) k_spmv<float><<<grid, kThreads, 0, s>>>(ptr, idx, val, tiles, ntiles, v, out, b, part);
    else k_spmv<double><<<grid, kThreads, 0, s>>>(ptr, idx, val, tiles, ntiles, v, out, b, part);
    return cudaGetLastError();
}

cudaError_t launch_colweights(const int32_t *ptr, const void *val, bool f32, int64_t n, int32_t mode,
                              double *w, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int grid = int((n + kThreads - 1) / kThreads);
    if (f32) k_colweights<float><<<grid, kThreads, 0, s>>>(ptr, val, n, mode, w);
    else k_colweights<double><<<grid, kThreads, 0, s>>>(ptr, val, n, mode, w);
    return cudaGetLastError();
}

}  // namespace plss
