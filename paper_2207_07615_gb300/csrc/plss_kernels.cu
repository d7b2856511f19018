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
// The update leaves its theta partials to the row sweep that follows: that
// sweep's finishing CTA sums them, records the update and then applies the
// stopping rule.
//
// Every nonzero of a sweep is one random gather of the dense operand, and
// on GB300 those gathers (about 250 G sectors/s) rather than HBM bytes set
// the time; the FP64 pipe runs at a small fraction of the FP32 rate, so FP64
// sweeps spend one FMA per nonzero and FP32 sweeps none. The kernels are
// plain CUDA-core code:
//   * sliced tiles (tiles of short segments, stored 32 slots wide, g lanes
//     per segment): the warp loads 32 consecutive indices and values per
//     step, 8 steps before their 8 gathers; a single system whose side is
//     sliced throughout runs that side over balanced warp ranges of slices
//     (k_row_sweep_w, k_col_sweep_w) with one partial per CTA;
//   * staged tiles (FP32, and FP64 tiles of uneven segments): products
//     staged in shared memory, summed there by G lanes per segment;
//   * CSR/CSC tiles (G lanes per segment, long segments one CTA each);
//   * per-tile (or per-CTA) FP64 partial sums of rho / phi / theta, summed in
//     a fixed order by the CTA that completes a system (deterministic for a
//     given schedule), which then takes the scalar step.
#include <cuda_runtime.h>

#include <type_traits>

#include "plss_dev.cuh"
#include "plss_devfn.cuh"
#include "plss_launch.h"

namespace plss {

constexpr int kBatch = 8;   // loads each lane issues before using any of them
// Steps of a column slice each lane loads before its gathers: four in FP64,
// eight in FP32 (C2's ~40-element columns: the FP64 column sweep takes
// 40.5 us with four and 42.0 us with eight; the FP32 one took 54.9 us with
// four against 38.3 us with eight).
template <typename S>
constexpr int kColBatch = std::is_same<S, double>::value ? 4 : 8;
constexpr int kWarpSweepCtas = 4;   // resident CTAs per SM of the warp-range sweeps

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// Fixed-order sum over the CTA of N doubles: a shuffle tree in every warp,
// then one over the warp totals. On GB300 a FP64 warp-instruction costs the
// same whether one lane or 32 are active, so full-warp trees (5 + 3
// dependent FP64 adds) beat sequential folds. Every thread calls it; the
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
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double t = lane < kWarps ? sh[i][lane] : 0.0;
#pragma unroll
            for (int o = kWarps / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[i] = t;
        }
    }
}

// Fixed-order CTA sum of N double-float values; the double result is valid
// in thread 0 (three FP64 operations per value, by one thread).
template <int N>
__device__ __forceinline__ void cta_sum_df(const DF (&v)[N], double (&out)[N]) {
    __shared__ float shh[N][kThreads], shl[N][kThreads];
    __shared__ DF sh2[N][32];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        shh[i][threadIdx.x] = v[i].hi;
        shl[i][threadIdx.x] = v[i].lo;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            DF t = {shh[i][threadIdx.x], shl[i][threadIdx.x]};
#pragma unroll
            for (int q = 1; q < kWarps; ++q)
                t = df_add(t, DF{shh[i][threadIdx.x + 32 * q], shl[i][threadIdx.x + 32 * q]});
            sh2[i][threadIdx.x] = t;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < N; ++i) {
            DF t = sh2[i][threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                t = df_add(t, DF{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)});
            if (threadIdx.x == 0) out[i] = double(t.hi) + double(t.lo);
        }
    }
}

// Dot product of one sparse segment (nonzeros [s, e)) with a dense vector,
// split over the G lanes of a group (lane gl takes s+gl, s+gl+G, ...); each
// lane issues 8 index/value loads, then their 8 gathers, then its 8 FMAs,
// so one FMA is spent per nonzero plus log2(G) tree levels per segment. The
// sum lands in every lane of the group. All 32 lanes of the warp must call
// it (warp-uniform control flow around the call).
template <int G, typename VT, typename XT, typename ACC>
__device__ __forceinline__ ACC seg_dot(const int32_t *__restrict__ idx, const VT *__restrict__ val,
                                       int32_t s, int32_t e, int gl, const XT *__restrict__ x) {
    ACC acc = ACC(0);
    for (int32_t base = s + gl; base < e; base += kBatch * G) {
        int32_t c[kBatch];
        VT v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int32_t k = base + u * G;
            const bool in = k < e;
            c[u] = in ? __ldg(idx + k) : 0;
            v[u] = in ? __ldg(val + k) : VT(0);
        }
        XT g[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) g[u] = base + u * G < e ? __ldg(x + c[u]) : XT(0);
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (base + u * G < e) acc = fma_t(ACC(v[u]), ACC(g[u]), acc);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Dot product of one long segment [s, e) with a dense vector, streamed by
// the whole CTA in batches of 8 loads per thread; thread partials combined
// in a fixed order in double (result in thread 0).
template <typename VT, typename XT, typename ACC>
__device__ __forceinline__ double cta_dot(const int32_t *__restrict__ idx,
                                          const VT *__restrict__ val, int32_t s, int32_t e,
                                          const XT *__restrict__ x) {
    ACC acc = ACC(0);
    for (int32_t base = s + threadIdx.x; base < e; base += kBatch * kThreads) {
        int32_t c[kBatch];
        VT v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int32_t k = base + u * kThreads;
            const bool in = k < e;
            c[u] = in ? __ldg(idx + k) : 0;
            v[u] = in ? __ldg(val + k) : VT(0);
        }
        XT g[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) g[u] = base + u * kThreads < e ? __ldg(x + c[u]) : XT(0);
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (base + u * kThreads < e) acc = fma_t(ACC(v[u]), ACC(g[u]), acc);
    }
    double v1[1] = {double(acc)};
    cta_sum<1>(v1);
    return v1[0];
}

// Staged tiles (kSliced unset, kStaged set: every FP32 tile that is not
// sliced, and FP64 tiles of uneven segments): a tile's products are staged
// in shared memory. Every thread issues its (up to 8) coalesced index/value
// loads, the tile's segment offsets and (row sweep) old residuals, then its
// gathers, before storing any product; the segments are then summed out of
// shared memory by G lanes each, so a long segment among short ones costs
// shared-memory adds rather than a warp's serial gather chain.
constexpr int kStageNnz = 2048;                   // products staged per tile
constexpr int kStagePer = kStageNnz / kThreads;   // nonzeros per thread
constexpr int kStageSegs = 1024;                  // segments per staged tile (host: kTileMaxSegsF32)
constexpr int kStageSegPer = (kStageSegs + 1 + kThreads - 1) / kThreads;

template <typename T>
struct Stage {
    T prod[kStageNnz];
    int32_t ptr[kStageSegs + 1];
    T old[kStageSegs];
};

// Stages the tile [t.begin, t.end) of ptr/idx/val against x; with `vec`,
// also old[i] = vec[t.begin + i]. All global loads (indices, values,
// segment offsets, old values) are issued before any is used, then the
// gathers, then the shared-memory stores. Ends with __syncthreads().
template <typename T>
__device__ __forceinline__ void stage_tile(const Tile &t, const int32_t *__restrict__ ptr,
                                           const int32_t *__restrict__ idx, const T *__restrict__ val,
                                           const T *__restrict__ x, const T *__restrict__ vec, Stage<T> &sm) {
    const int32_t nseg = t.end - t.begin;
    const int32_t z0 = __ldg(ptr + t.begin);
    const int32_t nz = __ldg(ptr + t.end) - z0;
    int32_t c[kStagePer];
    T v[kStagePer];
#pragma unroll
    for (int u = 0; u < kStagePer; ++u) {
        const int32_t k = threadIdx.x + u * kThreads;
        const bool in = k < nz;
        c[u] = in ? __ldg(idx + z0 + k) : 0;
        v[u] = in ? __ldg(val + z0 + k) : T(0);
    }
    int32_t pq[kStageSegPer];
    T oq[kStageSegPer];
#pragma unroll
    for (int q = 0; q < kStageSegPer; ++q) {
        const int32_t i = threadIdx.x + q * kThreads;
        pq[q] = i <= nseg ? __ldg(ptr + t.begin + i) : 0;
        oq[q] = vec && i < nseg ? vec[t.begin + i] : T(0);
    }
    T g[kStagePer];
#pragma unroll
    for (int u = 0; u < kStagePer; ++u) g[u] = threadIdx.x + u * kThreads < nz ? __ldg(x + c[u]) : T(0);
#pragma unroll
    for (int q = 0; q < kStageSegPer; ++q) {
        const int32_t i = threadIdx.x + q * kThreads;
        if (i <= nseg) sm.ptr[i] = pq[q] - z0;
        if (i < nseg) sm.old[i] = oq[q];
    }
#pragma unroll
    for (int u = 0; u < kStagePer; ++u) {
        const int32_t k = threadIdx.x + u * kThreads;
        if (k < nz) sm.prod[k] = v[u] * g[u];
    }
    __syncthreads();
}

// Calls body(i, d, gl, valid) with d the sum over segment i of the tile
// (tile-local index), G lanes per segment; warp-uniform loop.
template <int G, typename T, typename F>
__device__ __forceinline__ void staged_segments(const Tile &t, const Stage<T> &sm, F &&body) {
    constexpr int SPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane & (G - 1);
    const int32_t nseg = t.end - t.begin;
    for (int32_t base = warp * SPW; base < nseg; base += kWarps * SPW) {
        const int32_t i = base + gid;
        const bool valid = i < nseg;
        const int32_t s = valid ? sm.ptr[i] : 0, e = valid ? sm.ptr[i + 1] : 0;
        T acc = T(0);
        for (int32_t k = s + gl; k < e; k += G) acc += sm.prod[k];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        body(i, acc, gl, valid);
    }
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

// Random gathers of the sliced sweeps: cached in L2 only (L1 would only
// take fills that are never reused).
template <typename T>
__device__ __forceinline__ T kGather(const T *p) { return __ldcg(p); }

// Loads of A's sliced index and value streams, each element read once per
// sweep: non-coherent, and not allocated in L1 (nothing there is read
// again). On C2 this took 2-4 % off a sweep against plain __ldg.
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream(const double *p) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

// Dot product of slot `lane` of a slice (element offset `off`, `width`
// elements per slot) with a dense vector: the warp loads 32 consecutive
// indices and values per step, B steps before their gathers, and each lane
// sums its own segment in element order with one FMA per element. Padding
// (index -1, value 0) gathers nothing and adds an exact zero.
template <typename VT, typename XT, typename ACC, int B = kBatch>
__device__ __forceinline__ ACC slice_dot(const int32_t *__restrict__ idx, const VT *__restrict__ val,
                                         int32_t off, int32_t width, int lane, const XT *__restrict__ x) {
    ACC acc = ACC(0);
    for (int32_t k0 = 0; k0 < width; k0 += B) {
        int32_t c[B];
        VT v[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const bool in = k0 + u < width;
            const int32_t e = off + 32 * (k0 + u) + lane;
            c[u] = in ? ld_stream(idx + e) : -1;
            v[u] = in ? ld_stream(val + e) : VT(0);
        }
        XT g[B];
#pragma unroll
        for (int u = 0; u < B; ++u) g[u] = c[u] >= 0 ? kGather(x + c[u]) : XT(0);
#pragma unroll
        for (int u = 0; u < B; ++u) acc = fma_t(ACC(v[u]), ACC(g[u]), acc);
    }
    return acc;
}

// Sum over the g lanes of a segment (g a power of two; every lane takes
// part; the same fixed order in every lane of the group).
template <typename T>
__device__ __forceinline__ T group_sum(T v, int g) {
    for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Calls body(seg, off, width, lane) for each slot of the sliced tile `ti`
// (one warp per slice; seg < 0 for an empty slot); warp-uniform loop.
template <typename F>
__device__ __forceinline__ void for_slices(const Sliced &sl, const Tile &t, int32_t ti, F &&body) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t s0 = __ldg(sl.first + ti);
    const int32_t per = 32 / sl.g;   // segments per slice
    const int32_t ns = (t.end - t.begin + per - 1) / per;
    for (int32_t s = warp; s < ns; s += kWarps) {
        const int32_t off = __ldg(sl.ptr + s0 + s);
        const int32_t width = (__ldg(sl.ptr + s0 + s + 1) - off) >> 5;
        const int32_t seg = __ldg(sl.seg + 32 * (s0 + s) + lane);
        body(seg, off, width, lane);
    }
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
                                         double &acc_r, double &acc_b) {
    const S *__restrict__ val = static_cast<const S *>(a.val);
    S *__restrict__ r = static_cast<S *>(a.r);
    if (init) {
        for_segments<G>(a.row_ptr, t, [&](int32_t row, int32_t s, int32_t e, int gl, bool valid) {
            const double d = seg_dot<G, S, double, double>(a.col_idx, val, s, e, gl, a.x);
            if (valid && gl == 0) {
                const double bi = a.b[row];
                const S ri = S(bi - d);
                r[row] = ri;
                acc_r = fma(double(ri), double(ri), acc_r);
                acc_b = fma(bi, bi, acc_b);
            }
        });
    } else {
        const S *__restrict__ p = static_cast<const S *>(a.p);
        for_segments<G>(a.row_ptr, t, [&](int32_t row, int32_t s, int32_t e, int gl, bool valid) {
            const S old = valid && gl == 0 ? r[row] : S(0);   // issued before the dot's loads
            const S d = seg_dot<G, S, S, S>(a.col_idx, val, s, e, gl, p);
            if (valid && gl == 0) {
                const S ri = old - d;
                r[row] = ri;
                acc_r = fma(double(ri), double(ri), acc_r);
            }
        });
    }
}

// r = r - A p on a staged tile; rho partial in double-float (FP32) or
// double (FP64).
template <int G, typename S>
__device__ __forceinline__ void row_tile_staged(const SweepArgs &a, const Tile &t, DF &acc_f, double &acc_d,
                                                unsigned char *stage) {
    S *__restrict__ r = static_cast<S *>(a.r);
    Stage<S> &sm = *reinterpret_cast<Stage<S> *>(stage);
    stage_tile<S>(t, a.row_ptr, a.col_idx, static_cast<const S *>(a.val), static_cast<const S *>(a.p), r, sm);
    staged_segments<G>(t, sm, [&](int32_t i, S d, int gl, bool valid) {
        if (valid && gl == 0) {
            const S ri = sm.old[i] - d;
            r[t.begin + i] = ri;
            if constexpr (std::is_same<S, float>::value) acc_f = df_add_prod(acc_f, ri, ri);
            else acc_d = fma(ri, ri, acc_d);
        }
    });
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
            acc_r = fma(double(ri), double(ri), acc_r);
            acc_b = fma(bi, bi, acc_b);
        } else {
            const S ri = r[row] - S(d);
            r[row] = ri;
            acc_r = fma(double(ri), double(ri), acc_r);
        }
    }
}

// One slot (row) of a slice in the row sweep: r = r - A p, or r = b - A x
// with products in double after a (re)start; rho (and ||b||^2) partials in
// double.
template <typename S>
__device__ __forceinline__ void row_slot(const SweepArgs &a, int32_t row, int32_t off, int32_t width,
                                         int lane, bool init, double &acc_r, double &acc_b) {
    const S *__restrict__ val = static_cast<const S *>(a.rsl.val);
    S *__restrict__ r = static_cast<S *>(a.r);
    const int g = a.rsl.g;
    const bool lead = row >= 0 && (lane & (g - 1)) == 0;   // first lane of the row's group
    if (init) {
        const double bi = lead ? a.b[row] : 0.0;
        const double d = group_sum(slice_dot<S, double, double>(a.rsl.idx, val, off, width, lane, a.x), g);
        if (lead) {
            const S ri = S(bi - d);
            r[row] = ri;
            acc_r = fma(double(ri), double(ri), acc_r);
            acc_b = fma(bi, bi, acc_b);
        }
    } else {
        const S old = lead ? r[row] : S(0);   // issued before the dot's loads
        const S d = group_sum(slice_dot<S, S, S>(a.rsl.idx, val, off, width, lane, static_cast<const S *>(a.p)), g);
        if (lead) {
            const S ri = old - d;
            r[row] = ri;
            acc_r = fma(double(ri), double(ri), acc_r);
        }
    }
}

// Sliced tile of the row sweep (both storage types); one lane per row.
template <typename S>
__device__ __forceinline__ void row_tile_sliced(const SweepArgs &a, const Tile &t, int32_t ti, bool init,
                                                double &acc_r, double &acc_b) {
    for_slices(a.rsl, t, ti, [&](int32_t row, int32_t off, int32_t width, int lane) {
        row_slot<S>(a, row, off, width, lane, init, acc_r, acc_b);
    });
}

// The stopping rule after a row sweep (one thread): rho = r^T r, and with
// `init` (r = b - A x) bb = ||b||^2.
__device__ void row_decide(const SweepArgs &a, SysState *st, bool init, double rho, double bb) {
    st->cnt_row = 0;
    if (init) {
        st->nb = sqrt(bb);
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
    } else {
        // the transition the recursion takes next
        int32_t next = PH_RUN, flags = 0;
        if (!init && st->inner_tol2 > 0.0 && (rho <= st->inner_tol2 * st->rho0 || rho > 4.0 * st->rho0)) {
            // inner solve done, or the float recursion has drifted upwards:
            // refine from b - A x
            next = PH_SETUP;
            flags = 0x10;
        } else if (init) {
            // after a refresh of r from b - A x: a new recursion, or (residual
            // replacement) the same one going on with the fresh residual
            next = (st->replace && !st->restart_next) ? PH_RUN : PH_FIRST;
            flags = 0x20;
        }
        if (st->iters >= st->maxit) {
            // the update cap: stop, keeping the transition for a resume
            st->resume = next | flags | 0x100;
            finish_system(a, st, 1);
        } else {
            if (flags & 0x10) st->since = 0;
            if (flags & 0x20) st->restart_next = 0;
            st->phase = next;
        }
    }
}

// After an update (one thread, in the row sweep's finishing CTA, before the
// stopping rule): theta = p^T W^{-1} p, the optional history row, the update
// count and the refinement counter.
__device__ void upd_done(SysState *st, double theta) {
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
    st->since = st->phase == PH_SETUP ? 0 : st->since + 1;
    st->upd = 0;
}

// Sums the row-sweep partials [pb, pb + pc) of system `sys` in a fixed order
// and applies the stopping rule (whole CTA; the last CTA of the system).
__device__ void finish_row(const SweepArgs &a, int32_t sys, bool init, int32_t pb, int32_t pc) {
    const SysDesc d = a.desc[sys];
    const bool upd = reinterpret_cast<const volatile int32_t *>(&a.st[sys].upd)[0] != 0;
    double v[3] = {0.0, 0.0, 0.0};
    for (int32_t i = threadIdx.x; i < pc; i += kThreads) {
        v[0] += __ldcg(a.part_row + 2 * (pb + i));
        v[1] += __ldcg(a.part_row + 2 * (pb + i) + 1);
    }
    if (upd)   // theta of the update this row sweep followed
        for (int32_t i = threadIdx.x; i < d.vt_count; i += kThreads) v[2] += __ldcg(a.part_upd + d.vt_begin + i);
    cta_sum<3>(v);
    if (threadIdx.x == 0) {
        SysState *st = a.st + sys;
        if (upd) upd_done(st, v[2]);
        row_decide(a, st, init, v[0], v[1]);
    }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_row_sweep(SweepArgs a) {
    __shared__ __align__(16) unsigned char stage[sizeof(Stage<S>)];   // staged tiles
    wait_prior_grid();
    int32_t t0, t1;
    tile_range(a.n_rtiles, t0, t1);
    int32_t cur = -1;
    uint32_t pending = 0;
    bool active = false, init = false;
    for (int32_t ti = t0; ti < t1; ++ti) {
        const Tile t = a.rtiles[ti];
        if (t.sys != cur) {
            if (pending && arrive(&a.st[cur].cnt_row, pending, a.desc[cur].rt_count))
                finish_row(a, cur, init, a.desc[cur].rt_begin, a.desc[cur].rt_count);
            cur = t.sys;
            pending = 0;
            const int32_t ph = load_phase(a.st + cur);
            active = ph == PH_SETUP || ph == PH_RUN;
            init = ph == PH_SETUP;
        }
        if (!active) continue;
        double acc[2] = {0.0, 0.0};
        if (t.group & kSliced) {
            row_tile_sliced<S>(a, t, ti, init, acc[0], acc[1]);
            cta_sum<2>(acc);
        } else if ((t.group & kStaged) && !init) {
            DF f[1] = {{0.0f, 0.0f}};
            switch (t.group & kGroupMask) {
                case 1: row_tile_staged<1, S>(a, t, f[0], acc[0], stage); break;
                case 2: row_tile_staged<2, S>(a, t, f[0], acc[0], stage); break;
                case 4: row_tile_staged<4, S>(a, t, f[0], acc[0], stage); break;
                case 8: row_tile_staged<8, S>(a, t, f[0], acc[0], stage); break;
                case 16: row_tile_staged<16, S>(a, t, f[0], acc[0], stage); break;
                default: row_tile_staged<32, S>(a, t, f[0], acc[0], stage); break;
            }
            if constexpr (std::is_same<S, float>::value) {
                double o[1];
                cta_sum_df<1>(f, o);
                acc[0] = o[0];
            } else {
                cta_sum<2>(acc);
            }
        } else {
            switch (t.group & kGroupMask) {
                case 0: row_tile_cta<S>(a, t, init, acc[0], acc[1]); break;
                case 1: row_tile<1, S>(a, t, init, acc[0], acc[1]); break;
                case 2: row_tile<2, S>(a, t, init, acc[0], acc[1]); break;
                case 4: row_tile<4, S>(a, t, init, acc[0], acc[1]); break;
                case 8: row_tile<8, S>(a, t, init, acc[0], acc[1]); break;
                case 16: row_tile<16, S>(a, t, init, acc[0], acc[1]); break;
                default: row_tile<32, S>(a, t, init, acc[0], acc[1]); break;
            }
            cta_sum<2>(acc);
        }
        if (threadIdx.x == 0) {
            a.part_row[2 * ti] = acc[0];
            a.part_row[2 * ti + 1] = acc[1];
        }
        ++pending;
    }
    if (pending && arrive(&a.st[cur].cnt_row, pending, a.desc[cur].rt_count))
        finish_row(a, cur, init, a.desc[cur].rt_begin, a.desc[cur].rt_count);
}

// Row sweep of a single-system context whose row tiles are all sliced: each
// warp takes one range of slices (Sliced::wr), one partial per CTA, one barrier per
// CTA (its closing sum) instead of one per tile.
template <typename S>
__global__ void __launch_bounds__(kThreads) k_row_sweep_w(SweepArgs a) {
    const int lane = threadIdx.x & 31;
    // warp k of CTA b takes range k * gridDim.x + b: a CTA's (and an SM's)
    // warps draw ranges from all along the length-sorted slices
    const int32_t w = int32_t(threadIdx.x >> 5) * int32_t(gridDim.x) + int32_t(blockIdx.x);
    const int32_t s0 = __ldg(a.rsl.wr + w), s1 = __ldg(a.rsl.wr + w + 1);
    wait_prior_grid();
    const int32_t ph = load_phase(a.st);
    if (ph != PH_SETUP && ph != PH_RUN) return;   // uniform over the grid
    const bool init = ph == PH_SETUP;
    double acc[2] = {0.0, 0.0};
    for (int32_t s = s0; s < s1; ++s) {
        const int32_t off = __ldg(a.rsl.ptr + s);
        const int32_t width = (__ldg(a.rsl.ptr + s + 1) - off) >> 5;
        const int32_t row = __ldg(a.rsl.seg + 32 * s + lane);
        row_slot<S>(a, row, off, width, lane, init, acc[0], acc[1]);
    }
    cta_sum<2>(acc);
    if (threadIdx.x == 0) {
        a.part_row[2 * blockIdx.x] = acc[0];
        a.part_row[2 * blockIdx.x + 1] = acc[1];
    }
    if (arrive(&a.st->cnt_row, 1, int32_t(gridDim.x))) finish_row(a, 0, init, 0, int32_t(gridDim.x));
}

// ---------------------------------------------------------------------------
// Column sweep: y = A^T r, u = W y, phi = y^T u, then the scalar step
// ---------------------------------------------------------------------------

template <typename S>
__device__ __forceinline__ void col_out(const SweepArgs &a, int32_t col, double y, double &acc) {
    const S uj = a.w ? S(a.w[col] * y) : S(y);
    static_cast<S *>(a.u)[col] = uj;
    acc = fma(y, double(uj), acc);
}

template <int G, typename S>
__device__ __forceinline__ void col_tile(const SweepArgs &a, const Tile &t, double &acc) {
    const S *__restrict__ val = static_cast<const S *>(a.cval);
    const S *__restrict__ r = static_cast<const S *>(a.r);
    for_segments<G>(a.col_ptr, t, [&](int32_t col, int32_t s, int32_t e, int gl, bool valid) {
        const S d = seg_dot<G, S, S, S>(a.row_idx, val, s, e, gl, r);
        if (valid && gl == 0) col_out<S>(a, col, double(d), acc);
    });
}

// y = A^T r on a staged tile, u = W y (float weights for FP32 storage), phi
// partial in double-float (FP32) or double (FP64).
template <int G, typename S>
__device__ __forceinline__ void col_tile_staged(const SweepArgs &a, const Tile &t, DF &acc_f, double &acc_d,
                                                unsigned char *stage) {
    Stage<S> &sm = *reinterpret_cast<Stage<S> *>(stage);
    S *__restrict__ u = static_cast<S *>(a.u);
    stage_tile<S>(t, a.col_ptr, a.row_idx, static_cast<const S *>(a.cval), static_cast<const S *>(a.r), nullptr, sm);
    staged_segments<G>(t, sm, [&](int32_t i, S y, int gl, bool valid) {
        if (valid && gl == 0) {
            const int32_t col = t.begin + i;
            if constexpr (std::is_same<S, float>::value) {
                const float uj = a.wf ? __fmul_rn(a.wf[col], y) : y;
                u[col] = uj;
                acc_f = df_add_prod(acc_f, y, uj);
            } else {
                col_out<S>(a, col, y, acc_d);
            }
        }
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

// One slot (column) of a slice in the column sweep: y = A^T r, u = W y
// (float weights for FP32 storage), phi partial in double.
template <typename S>
__device__ __forceinline__ void col_slot(const SweepArgs &a, int32_t col, int32_t off, int32_t width,
                                         int lane, double &acc) {
    const int g = a.csl.g;
    const S y = group_sum(slice_dot<S, S, S, kColBatch<S>>(a.csl.idx, static_cast<const S *>(a.csl.val), off, width,
                                                           lane, static_cast<const S *>(a.r)), g);
    if (col >= 0 && (lane & (g - 1)) == 0) {
        if constexpr (std::is_same<S, float>::value) {
            const float uj = a.wf ? __fmul_rn(a.wf[col], y) : y;
            static_cast<float *>(a.u)[col] = uj;
            acc = fma(double(y), double(uj), acc);
        } else {
            col_out<S>(a, col, double(y), acc);
        }
    }
}

// Sliced tile of the column sweep; one lane per column.
template <typename S>
__device__ __forceinline__ void col_tile_sliced(const SweepArgs &a, const Tile &t, int32_t ti, double &acc) {
    for_slices(a.csl, t, ti, [&](int32_t col, int32_t off, int32_t width, int lane) {
        col_slot<S>(a, col, off, width, lane, acc);
    });
}

// The scalar step of Theorem 4.1 after a column sweep (one thread): phi =
// y^T W y gives beta and gamma (or the first update's gamma = rho/phi), or a
// breakdown.
__device__ void col_decide(const SweepArgs &a, SysState *st, double phi) {
    st->cnt_col = 0;
    st->phi = phi;
    const double rho = st->rho;
    const bool first = st->phase == PH_FIRST;
    if (first) {
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
                st->restart_next = 1;
            } else {
                finish_system(a, st, -4);
            }
            return;
        }
        const double beta = __ddiv_rn(1.0, dd);
        st->beta = beta;
        st->gamma = __dmul_rn(__ddiv_rn(theta, rho), beta);
    }
    // the update of this body is due; the row sweep that follows it sees
    // PH_RUN, or PH_SETUP when the periodic refinement restarts from b - A x
    st->upd = first ? 2 : 1;
    st->phase = (st->refine > 0 && st->since + 1 >= st->refine) ? PH_SETUP : PH_RUN;
}

// Sums the column-sweep partials [pb, pb + pc) of system `sys` in a fixed
// order and takes the scalar step (whole CTA; the last CTA of the system).
__device__ void finish_col(const SweepArgs &a, int32_t sys, int32_t pb, int32_t pc) {
    double v[1] = {0.0};
    for (int32_t i = threadIdx.x; i < pc; i += kThreads) v[0] += __ldcg(a.part_col + pb + i);
    cta_sum<1>(v);
    if (threadIdx.x == 0) col_decide(a, a.st + sys, v[0]);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_col_sweep(SweepArgs a) {
    __shared__ __align__(16) unsigned char stage[sizeof(Stage<S>)];   // staged tiles
    wait_prior_grid();
    int32_t t0, t1;
    tile_range(a.n_ctiles, t0, t1);
    int32_t cur = -1;
    uint32_t pending = 0;
    bool active = false;
    for (int32_t ti = t0; ti < t1; ++ti) {
        const Tile t = a.ctiles[ti];
        if (t.sys != cur) {
            if (pending && arrive(&a.st[cur].cnt_col, pending, a.desc[cur].ct_count))
                finish_col(a, cur, a.desc[cur].ct_begin, a.desc[cur].ct_count);
            cur = t.sys;
            pending = 0;
            const int32_t ph = load_phase(a.st + cur);
            active = ph == PH_FIRST || ph == PH_RUN;
        }
        if (!active) continue;
        double acc[1] = {0.0};
        if (t.group & kSliced) {
            col_tile_sliced<S>(a, t, ti, acc[0]);
            cta_sum<1>(acc);
        } else if (t.group & kStaged) {
            DF f[1] = {{0.0f, 0.0f}};
            switch (t.group & kGroupMask) {
                case 1: col_tile_staged<1, S>(a, t, f[0], acc[0], stage); break;
                case 2: col_tile_staged<2, S>(a, t, f[0], acc[0], stage); break;
                case 4: col_tile_staged<4, S>(a, t, f[0], acc[0], stage); break;
                case 8: col_tile_staged<8, S>(a, t, f[0], acc[0], stage); break;
                case 16: col_tile_staged<16, S>(a, t, f[0], acc[0], stage); break;
                default: col_tile_staged<32, S>(a, t, f[0], acc[0], stage); break;
            }
            if constexpr (std::is_same<S, float>::value) cta_sum_df<1>(f, acc);
            else cta_sum<1>(acc);
        } else {
            switch (t.group & kGroupMask) {
                case 0: col_tile_cta<S>(a, t, acc[0]); break;
                case 1: col_tile<1, S>(a, t, acc[0]); break;
                case 2: col_tile<2, S>(a, t, acc[0]); break;
                case 4: col_tile<4, S>(a, t, acc[0]); break;
                case 8: col_tile<8, S>(a, t, acc[0]); break;
                case 16: col_tile<16, S>(a, t, acc[0]); break;
                default: col_tile<32, S>(a, t, acc[0]); break;
            }
            cta_sum<1>(acc);
        }
        if (threadIdx.x == 0) a.part_col[ti] = acc[0];
        ++pending;
    }
    if (pending && arrive(&a.st[cur].cnt_col, pending, a.desc[cur].ct_count))
        finish_col(a, cur, a.desc[cur].ct_begin, a.desc[cur].ct_count);
}

// Column sweep of a single-system context whose column tiles are all
// sliced (warp ranges as in k_row_sweep_w).
template <typename S>
__global__ void __launch_bounds__(kThreads) k_col_sweep_w(SweepArgs a) {
    const int lane = threadIdx.x & 31;
    // warp k of CTA b takes range k * gridDim.x + b: a CTA's (and an SM's)
    // warps draw ranges from all along the length-sorted slices
    const int32_t w = int32_t(threadIdx.x >> 5) * int32_t(gridDim.x) + int32_t(blockIdx.x);
    const int32_t s0 = __ldg(a.csl.wr + w), s1 = __ldg(a.csl.wr + w + 1);
    wait_prior_grid();
    const int32_t ph = load_phase(a.st);
    if (ph != PH_FIRST && ph != PH_RUN) return;   // uniform over the grid
    double acc[1] = {0.0};
    for (int32_t s = s0; s < s1; ++s) {
        const int32_t off = __ldg(a.csl.ptr + s);
        const int32_t width = (__ldg(a.csl.ptr + s + 1) - off) >> 5;
        const int32_t col = __ldg(a.csl.seg + 32 * s + lane);
        col_slot<S>(a, col, off, width, lane, acc[0]);
    }
    cta_sum<1>(acc);
    if (threadIdx.x == 0) a.part_col[blockIdx.x] = acc[0];
    if (arrive(&a.st->cnt_col, 1, int32_t(gridDim.x))) finish_col(a, 0, 0, int32_t(gridDim.x));
}

// ---------------------------------------------------------------------------
// Update: p = beta p + gamma u, theta = p^T W^{-1} p, x = x + p
// ---------------------------------------------------------------------------

constexpr int kUpdU = 4;   // entries per thread in one pass (a pass covers 1,024 entries: one tile)

// The entries one thread updates in a pass (base, base + kThreads, ...).
template <typename S>
struct UpdRegs {
    using W = typename std::conditional<std::is_same<S, float>::value, float, double>::type;
    S u[kUpdU], p[kUpdU];
    double x[kUpdU];
    W w[kUpdU];
};

// Loads u, p, x and the weights of a pass (all of them, before any is
// used: one memory round trip). p is loaded on the first update too, and
// not used there.
template <typename S>
__device__ __forceinline__ void upd_load(const SweepArgs &a, int32_t base, int32_t end, UpdRegs<S> &g) {
    using W = typename UpdRegs<S>::W;
    const S *__restrict__ p = static_cast<const S *>(a.p);
    const S *__restrict__ u = static_cast<const S *>(a.u);
    const W *__restrict__ winv;
    if constexpr (std::is_same<S, float>::value) winv = a.winvf;
    else winv = a.winv;
#pragma unroll
    for (int q = 0; q < kUpdU; ++q) {
        const int32_t j = base + q * kThreads;
        const bool in = j < end;
        g.u[q] = in ? u[j] : S(0);
        g.p[q] = in ? p[j] : S(0);
        g.x[q] = in ? a.x[j] : 0.0;
        g.w[q] = in && winv ? winv[j] : W(1);
    }
}

// FP32 storage: p = beta p + gamma u in float (p is stored in float; beta
// and gamma rounded to float), theta partials in float per thread, x in
// double -- two FP64-pipe operations per entry.
__device__ __forceinline__ void upd_pass_f32(const SweepArgs &a, int32_t base, int32_t end, bool first,
                                             double beta, double gamma, const UpdRegs<float> &g, DF &acc) {
    float *__restrict__ p = static_cast<float *>(a.p);
    const bool weighted = a.winvf != nullptr;
    const float bf = float(beta), gf = float(gamma);
#pragma unroll
    for (int q = 0; q < kUpdU; ++q) {
        const int32_t j = base + q * kThreads;
        if (j < end) {
            const float pn = first ? gf * g.u[q] : fmaf(bf, g.p[q], gf * g.u[q]);
            p[j] = pn;
            acc = df_add_prod(acc, pn, weighted ? __fmul_rn(pn, g.w[q]) : pn);
            a.x[j] = g.x[q] + double(pn);
        }
    }
}

template <typename S>
__device__ __forceinline__ void upd_pass(const SweepArgs &a, int32_t base, int32_t end, bool first, double beta,
                                         double gamma, const UpdRegs<S> &g, double &acc) {
    S *__restrict__ p = static_cast<S *>(a.p);
    const bool weighted = a.winv != nullptr;
#pragma unroll
    for (int q = 0; q < kUpdU; ++q) {
        const int32_t j = base + q * kThreads;
        if (j < end) {
            const double gu = gamma * double(g.u[q]);
            const double pn = first ? gu : fma(beta, double(g.p[q]), gu);
            const S ps = S(pn);
            p[j] = ps;
            const double pd = double(ps);
            acc = fma(pd, weighted ? pd * double(g.w[q]) : pd, acc);
            a.x[j] = g.x[q] + pd;
        }
    }
}

// The update writes one theta partial per tile and finishes nothing: the
// row sweep that follows sums them (it has to wait for the whole update
// anyway), which takes the arrival and the last-CTA reduction off this
// short kernel's critical path. The tile list is fixed for the context, so
// the first tile is read before the wait; a tile's vector entries are then
// requested together with its system's scalars (they do not depend on
// them), so the kernel's work after the wait is a single memory round trip
// before the arithmetic.
template <typename S>
__global__ void __launch_bounds__(kThreads) k_update(SweepArgs a) {
    int32_t t0, t1;
    tile_range(a.n_vtiles, t0, t1);
    Tile t = t0 < t1 ? a.vtiles[t0] : Tile{0, 0, 0, 0};
    wait_prior_grid();
    int32_t cur = -1;
    bool active = false, first = false;
    double beta = 0.0, gamma = 0.0;
    for (int32_t ti = t0; ti < t1; ++ti) {
        if (ti > t0) t = a.vtiles[ti];
        const int32_t base0 = t.begin + int32_t(threadIdx.x);
        UpdRegs<S> g;
        upd_load<S>(a, base0, t.end, g);
        if (t.sys != cur) {
            cur = t.sys;
            const int32_t upd = reinterpret_cast<const volatile int32_t *>(&a.st[cur].upd)[0];
            active = upd != 0;
            first = upd == 2;
            beta = a.st[cur].beta;
            gamma = a.st[cur].gamma;
        }
        if (!active) continue;
        double acc[1];
        if constexpr (std::is_same<S, float>::value) {
            DF f[1] = {{0.0f, 0.0f}};
            for (int32_t base = base0; base < t.end; base += kThreads * kUpdU) {
                if (base != base0) upd_load<S>(a, base, t.end, g);
                upd_pass_f32(a, base, t.end, first, beta, gamma, g, f[0]);
            }
            cta_sum_df<1>(f, acc);
        } else {
            acc[0] = 0.0;
            for (int32_t base = base0; base < t.end; base += kThreads * kUpdU) {
                if (base != base0) upd_load<S>(a, base, t.end, g);
                upd_pass<S>(a, base, t.end, first, beta, gamma, g, acc[0]);
            }
            cta_sum<1>(acc);
        }
        if (threadIdx.x == 0) a.part_upd[ti] = acc[0];
    }
}

// ---------------------------------------------------------------------------
// Small systems: one thread-block cluster runs the whole recursion
// ---------------------------------------------------------------------------
//
// For a system of a few thousand rows a body of three grid-wide launches is
// all latency (kernel boundaries, arrivals, last-CTA reductions). Here a
// cluster of kClusterCtas CTAs per system runs the same body -- column sweep,
// scalar step, update, row sweep, stopping rule, in the same order and with
// the same decision functions -- for up to `bodies` bodies per launch. Each
// CTA owns a contiguous share of the rows and of the columns (balanced by
// nonzeros); after each phase it puts its fixed-order partial sum in its
// shared memory and the cluster meets at a hardware barrier
// (barrier.cluster, release/acquire: the phase's vector writes are then
// visible to the whole cluster); every CTA then reads the kClusterCtas
// partials through distributed shared memory in rank order and takes the
// same scalar decisions on its own copy of the system state, so no
// broadcast is needed. The vectors live in global memory (L2-resident);
// when the system is small enough (RES), every CTA also keeps whole copies
// of the two gathered vectors -- r for the column sweep, p for the row
// sweep -- in its shared memory, and the CTA that produces an entry writes it
// into all the cluster's copies (st.shared::cluster) before the phase's
// barrier, so that every gather is a shared-memory load instead of an L2
// round trip. The arithmetic and its order are the same in both forms.

constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 512;
constexpr int kClusterWarps = kClusterThreads / 32;

template <int N>
__device__ __forceinline__ void clu_block_sum(double (&v)[N]) {
    __shared__ double sh[N][kClusterWarps];
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
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double t = lane < kClusterWarps ? sh[i][lane] : 0.0;
#pragma unroll
            for (int o = kClusterWarps / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            v[i] = t;
        }
    }
}

// Cluster-wide barrier (hardware; release/acquire at cluster scope).
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Reads a double from the shared memory of CTA `rank` of this cluster.
__device__ __forceinline__ double dsmem_load(const double *p, uint32_t rank) {
    uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p)), remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
    return v;
}

// Writes v to the element `p` (this CTA's shared memory) of every CTA of
// the cluster, this one included.
template <typename T>
__device__ __forceinline__ void dsmem_store_all(T *p, T v) {
    const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p));
#pragma unroll
    for (uint32_t k = 0; k < uint32_t(kClusterCtas); ++k) {
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(k));
        if constexpr (sizeof(T) == 8)
            asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(double(v)) : "memory");
        else
            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(remote), "f"(float(v)) : "memory");
    }
}

// First segment of share k of [b0, b1) when the shares hold about equal
// nonzeros (offsets in ptr).
__device__ __forceinline__ int32_t clu_split(const int32_t *ptr, int32_t b0, int32_t b1, int k) {
    if (k <= 0) return b0;
    if (k >= kClusterCtas) return b1;
    const int64_t z0 = ptr[b0], z1 = ptr[b1];
    const int64_t goal = z0 + (z1 - z0) * k / kClusterCtas;
    int32_t lo = b0, hi = b1;   // first segment whose start is >= goal
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (ptr[mid] < goal) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int G, typename F>
__device__ __forceinline__ void clu_segments(const int32_t *__restrict__ ptr, int32_t b0, int32_t b1, F &&body) {
    constexpr int SPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane & (G - 1);
    for (int32_t base = b0 + warp * SPW; base < b1; base += kClusterWarps * SPW) {
        const int32_t seg = base + gid;
        const bool valid = seg < b1;
        const int32_t s = valid ? __ldg(ptr + seg) : 0;
        const int32_t e = valid ? __ldg(ptr + seg + 1) : 0;
        body(seg, s, e, gl, valid);
    }
}

// Segment dot with G lanes against a vector written within this kernel:
// x[c - off] from this CTA's shared-memory copy (SH), else coherent loads
// of x[c] from global memory.
template <int G, typename VT, typename XT, typename ACC, bool SH = false>
__device__ __forceinline__ ACC clu_dot(const int32_t *__restrict__ idx, const VT *__restrict__ val, int32_t s,
                                       int32_t e, int gl, const XT *x, int32_t off = 0) {
    ACC acc = ACC(0);
    for (int32_t base = s + gl; base < e; base += kBatch * G) {
        int32_t c[kBatch];
        VT v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int32_t k = base + u * G;
            const bool in = k < e;
            c[u] = in ? __ldg(idx + k) : 0;
            v[u] = in ? __ldg(val + k) : VT(0);
        }
        XT g[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if constexpr (SH) g[u] = base + u * G < e ? x[c[u] - off] : XT(0);
            else g[u] = base + u * G < e ? __ldcg(x + c[u]) : XT(0);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (base + u * G < e) acc = fma_t(ACC(v[u]), ACC(g[u]), acc);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// The shared-memory copies of the RES form: r of the system's rows (offset
// R0) and p of its columns (offset C0); null pointers in the plain form.
template <typename S>
struct CluVecs {
    S *r = nullptr, *p = nullptr;
    int32_t R0 = 0, C0 = 0;
};

template <int G, typename S, bool RES>
__device__ __forceinline__ void clu_row(const SweepArgs &a, int32_t r0, int32_t r1, bool init, double &acc_r,
                                        double &acc_b, const CluVecs<S> &sv) {
    const S *__restrict__ val = static_cast<const S *>(a.val);
    S *r = static_cast<S *>(a.r);
    clu_segments<G>(a.row_ptr, r0, r1, [&](int32_t row, int32_t s, int32_t e, int gl, bool valid) {
        if (init) {
            const double d = clu_dot<G, S, double, double>(a.col_idx, val, s, e, gl, a.x);
            if (valid && gl == 0) {
                const double bi = a.b[row];
                const S ri = S(bi - d);
                r[row] = ri;
                if constexpr (RES) dsmem_store_all(sv.r + (row - sv.R0), ri);
                acc_r = fma(double(ri), double(ri), acc_r);
                acc_b = fma(bi, bi, acc_b);
            }
        } else {
            S d;
            if constexpr (RES) d = clu_dot<G, S, S, S, true>(a.col_idx, val, s, e, gl, sv.p, sv.C0);
            else d = clu_dot<G, S, S, S>(a.col_idx, val, s, e, gl, static_cast<const S *>(a.p));
            if (valid && gl == 0) {
                const S ri = (RES ? sv.r[row - sv.R0] : r[row]) - d;
                r[row] = ri;
                if constexpr (RES) dsmem_store_all(sv.r + (row - sv.R0), ri);
                acc_r = fma(double(ri), double(ri), acc_r);
            }
        }
    });
}

template <int G, typename S, bool RES>
__device__ __forceinline__ void clu_col(const SweepArgs &a, int32_t c0, int32_t c1, double &acc,
                                        const CluVecs<S> &sv) {
    const S *__restrict__ val = static_cast<const S *>(a.cval);
    clu_segments<G>(a.col_ptr, c0, c1, [&](int32_t col, int32_t s, int32_t e, int gl, bool valid) {
        S y;
        if constexpr (RES) y = clu_dot<G, S, S, S, true>(a.row_idx, val, s, e, gl, sv.r, sv.R0);
        else y = clu_dot<G, S, S, S>(a.row_idx, val, s, e, gl, static_cast<const S *>(a.r));
        if (valid && gl == 0) {
            if constexpr (std::is_same<S, float>::value) {
                const float uj = a.wf ? __fmul_rn(a.wf[col], y) : y;
                static_cast<float *>(a.u)[col] = uj;
                acc = fma(double(y), double(uj), acc);
            } else {
                col_out<S>(a, col, double(y), acc);
            }
        }
    });
}

// Lanes per segment for a mean segment length (as the host's tile groups).
__device__ __forceinline__ int clu_group(int64_t nnz, int64_t segs) {
    int g = 1;
    while (g < 32 && 2 * g * 8 * segs <= nnz) g <<= 1;
    return g;
}

template <typename S, bool RES>
__global__ void __launch_bounds__(kClusterThreads) k_cluster_solve(SweepArgs a, int32_t bodies) {
    extern __shared__ __align__(16) unsigned char clu_dyn[];   // RES: r copy, then p copy
    __shared__ SysState sst;           // this CTA's copy of the system state
    // this CTA's partials (phi, theta, rho, ||b||^2), one set per parity of
    // the body: a CTA rewrites a set only after a barrier that every CTA
    // reaches after reading it
    __shared__ double parts[2][4];
    __shared__ int32_t done_local;     // stands in for the active count in CTAs other than rank 0
    const uint32_t rank = cluster_rank();
    const int32_t sys = int32_t(blockIdx.x) / kClusterCtas;
    const SysDesc d = a.desc[sys];
    const int32_t R0 = int32_t(d.row_off), R1 = R0 + d.m, C0 = int32_t(d.col_off), C1 = C0 + d.n;
    const int32_t r0 = clu_split(a.row_ptr, R0, R1, int(rank)), r1 = clu_split(a.row_ptr, R0, R1, int(rank) + 1);
    const int32_t c0 = clu_split(a.col_ptr, C0, C1, int(rank)), c1 = clu_split(a.col_ptr, C0, C1, int(rank) + 1);
    const int64_t nnz = int64_t(a.row_ptr[R1]) - a.row_ptr[R0];
    const int gr = clu_group(nnz, d.m), gc = clu_group(nnz, d.n);
    // only rank 0 changes global state (the active count, the history)
    SweepArgs al = a;
    if (threadIdx.x == 0) {
        sst = a.st[sys];
        done_local = 0;
        if (rank != 0) sst.hist = nullptr;
    }
    if (rank != 0) al.n_active = &done_local;
    CluVecs<S> sv;
    if constexpr (RES) {
        sv.r = reinterpret_cast<S *>(clu_dyn);
        sv.p = sv.r + d.m;
        sv.R0 = R0;
        sv.C0 = C0;
        const S *gr_ = static_cast<const S *>(a.r);
        const S *gp_ = static_cast<const S *>(a.p);
        for (int32_t i = threadIdx.x; i < d.m; i += kClusterThreads) sv.r[i] = __ldcg(gr_ + R0 + i);
        for (int32_t j = threadIdx.x; j < d.n; j += kClusterThreads) sv.p[j] = __ldcg(gp_ + C0 + j);
        // no CTA writes into another's copies before that one has loaded them
        cluster_barrier();
    }
    __syncthreads();
    SysState *st = &sst;
    // sum of partial q over the cluster, in rank order (the same in every CTA)
    auto cluster_total = [&](const double *part, int q) {
        double t = 0.0;
        for (uint32_t k = 0; k < uint32_t(kClusterCtas); ++k) t += dsmem_load(&part[q], k);
        return t;
    };
    for (int32_t it = 0; it < bodies; ++it) {
        __syncthreads();
        double *part = parts[it & 1];
        int32_t ph = st->phase;
        if (ph == PH_DONE) break;   // the same in every CTA of the cluster
        if (ph == PH_FIRST || ph == PH_RUN) {
            double w1[1] = {0.0};
            switch (gc) {
                case 1: clu_col<1, S, RES>(al, c0, c1, w1[0], sv); break;
                case 2: clu_col<2, S, RES>(al, c0, c1, w1[0], sv); break;
                case 4: clu_col<4, S, RES>(al, c0, c1, w1[0], sv); break;
                case 8: clu_col<8, S, RES>(al, c0, c1, w1[0], sv); break;
                case 16: clu_col<16, S, RES>(al, c0, c1, w1[0], sv); break;
                default: clu_col<32, S, RES>(al, c0, c1, w1[0], sv); break;
            }
            clu_block_sum<1>(w1);
            if (threadIdx.x == 0) part[0] = w1[0];
            cluster_barrier();   // u, phi partials complete
            if (threadIdx.x == 0) col_decide(al, st, cluster_total(part, 0));
            __syncthreads();
            if (st->upd != 0) {
                const bool first = st->upd == 2;
                const double beta = st->beta, gamma = st->gamma;
                double acc[1] = {0.0};
                S *p = static_cast<S *>(a.p);
                const S *u = static_cast<const S *>(a.u);
                for (int32_t j = c0 + threadIdx.x; j < c1; j += kClusterThreads) {
                    S ps;
                    const S pj = first ? S(0) : (RES ? sv.p[j - C0] : p[j]);
                    if constexpr (std::is_same<S, float>::value) {
                        const float bf = float(beta), gf = float(gamma);
                        ps = first ? gf * u[j] : fmaf(bf, pj, gf * u[j]);
                    } else {
                        const double gu = gamma * u[j];
                        ps = first ? gu : fma(beta, pj, gu);
                    }
                    p[j] = ps;
                    if constexpr (RES) dsmem_store_all(sv.p + (j - C0), ps);
                    const double pd = double(ps);
                    if constexpr (std::is_same<S, float>::value)
                        acc[0] = fma(pd, a.winvf ? double(__fmul_rn(ps, a.winvf[j])) : pd, acc[0]);
                    else
                        acc[0] = fma(pd, a.winv ? pd * a.winv[j] : pd, acc[0]);
                    a.x[j] = a.x[j] + pd;
                }
                clu_block_sum<1>(acc);
                if (threadIdx.x == 0) part[1] = acc[0];
                cluster_barrier();   // p, x, theta partials complete
                if (threadIdx.x == 0) upd_done(st, cluster_total(part, 1));
            }
            __syncthreads();
            ph = st->phase;
        }
        if (ph == PH_SETUP || ph == PH_RUN) {
            const bool init = ph == PH_SETUP;
            double w2[2] = {0.0, 0.0};
            switch (gr) {
                case 1: clu_row<1, S, RES>(al, r0, r1, init, w2[0], w2[1], sv); break;
                case 2: clu_row<2, S, RES>(al, r0, r1, init, w2[0], w2[1], sv); break;
                case 4: clu_row<4, S, RES>(al, r0, r1, init, w2[0], w2[1], sv); break;
                case 8: clu_row<8, S, RES>(al, r0, r1, init, w2[0], w2[1], sv); break;
                case 16: clu_row<16, S, RES>(al, r0, r1, init, w2[0], w2[1], sv); break;
                default: clu_row<32, S, RES>(al, r0, r1, init, w2[0], w2[1], sv); break;
            }
            clu_block_sum<2>(w2);
            if (threadIdx.x == 0) {
                part[2] = w2[0];
                part[3] = w2[1];
            }
            cluster_barrier();   // r, rho partials complete
            if (threadIdx.x == 0) row_decide(al, st, init, cluster_total(part, 2), cluster_total(part, 3));
        }
    }
    __syncthreads();
    // no CTA may exit while another can still read its shared memory
    cluster_barrier();
    if (rank == 0 && threadIdx.x == 0) a.st[sys] = sst;
}

// ---------------------------------------------------------------------------
// One system on the whole GPU, whole updates per launch (schedule COOP)
// ---------------------------------------------------------------------------
//
// The three sweeps of an update as phases of one cooperative kernel: the
// column sweep and the row sweep over the sliced sides with this grid's own
// warp ranges, the update over contiguous column ranges. Phases meet at grid
// barriers (a counter and a generation word; every wait is limited to 2 s,
// after which the CTA sets the error word and returns, and so do the others).
// After a barrier every CTA sums the phase's per-CTA partials in CTA order
// and takes the scalar step on its own shared-memory copy of the state, so
// all CTAs hold the same bits and no CTA finishes alone; CTA 0 alone writes
// the global state, the history and the active count. Vectors written by
// another CTA within the launch (u, p, r, x gathered) are read through L2.

constexpr unsigned long long kCoopWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long coop_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool coop_barrier(uint32_t *bar, int *sh_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *vb = bar;
        int ok = vb[2] == 0;
        if (ok) {
            const uint32_t gen = vb[1];
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                bar[0] = 0;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const unsigned long long t0 = coop_now();
                while (vb[1] == gen) {
                    if (vb[2] != 0) { ok = 0; break; }
                    if (coop_now() - t0 > kCoopWaitNs) {
                        atomicExch(bar + 2, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(20);
                }
            }
            __threadfence();
        }
        *sh_ok = ok;
    }
    __syncthreads();
    return *sh_ok != 0;
}

// Sum of part[0..G) in CTA order (every CTA the same), valid in thread 0.
__device__ __forceinline__ double coop_total(const double *part, int stride, int off) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < int(gridDim.x); i += kThreads) v[0] += __ldcg(part + stride * i + off);
    cta_sum<1>(v);
    return v[0];
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_coop_solve(SweepArgs a, const int32_t *rwr, const int32_t *cwr,
                                                         double *part, uint32_t *bar, int32_t bodies) {
    __shared__ SysState sst;
    __shared__ int32_t done_local;
    __shared__ int sh_ok;
    const int lane = threadIdx.x & 31;
    const int G = int(gridDim.x), bid = int(blockIdx.x);
    const int32_t w = int32_t(bid) * kWarps + (threadIdx.x >> 5);
    const int32_t n = a.desc[0].n;
    const int32_t j0 = int32_t(int64_t(n) * bid / G), j1 = int32_t(int64_t(n) * (bid + 1) / G);
    double *p_phi = part, *p_th = part + G, *p_rho = part + 2 * G;   // p_rho: pairs (rho, ||b||^2)
    SweepArgs al = a;
    if (threadIdx.x == 0) {
        sst = a.st[0];
        done_local = 0;
        if (bid != 0) sst.hist = nullptr;
    }
    if (bid != 0) al.n_active = &done_local;
    __syncthreads();
    SysState *st = &sst;
    for (int32_t it = 0; it < bodies; ++it) {
        __syncthreads();
        int32_t ph = st->phase;
        if (ph == PH_DONE) break;   // the same in every CTA
        if (ph == PH_FIRST || ph == PH_RUN) {
            double v[1] = {0.0};
            for (int32_t sl = __ldg(cwr + w); sl < __ldg(cwr + w + 1); ++sl) {
                const int32_t off = __ldg(a.csl.ptr + sl);
                const int32_t width = (__ldg(a.csl.ptr + sl + 1) - off) >> 5;
                col_slot<S>(al, __ldg(a.csl.seg + 32 * sl + lane), off, width, lane, v[0]);
            }
            cta_sum<1>(v);
            if (threadIdx.x == 0) p_phi[bid] = v[0];
            if (!coop_barrier(bar, &sh_ok)) return;
            const double phi = coop_total(p_phi, 1, 0);
            if (threadIdx.x == 0) col_decide(al, st, phi);
            __syncthreads();
            if (st->upd != 0) {
                const bool first = st->upd == 2;
                const double beta = st->beta, gamma = st->gamma;
                S *p = static_cast<S *>(a.p);
                const S *u = static_cast<const S *>(a.u);
                double th[1] = {0.0};
                if constexpr (std::is_same<S, float>::value) {
                    const float bf = float(beta), gf = float(gamma);
                    DF acc[1] = {{0.0f, 0.0f}};
                    for (int32_t j = j0 + threadIdx.x; j < j1; j += kThreads) {
                        const float uj = __ldcg(u + j);
                        const float pn = first ? gf * uj : fmaf(bf, p[j], gf * uj);
                        p[j] = pn;
                        acc[0] = df_add_prod(acc[0], pn, a.winvf ? __fmul_rn(pn, a.winvf[j]) : pn);
                        a.x[j] = a.x[j] + double(pn);
                    }
                    cta_sum_df<1>(acc, th);
                } else {
                    for (int32_t j = j0 + threadIdx.x; j < j1; j += kThreads) {
                        const double gu = gamma * double(__ldcg(u + j));
                        const double pn = first ? gu : fma(beta, double(p[j]), gu);
                        const S ps = S(pn);
                        p[j] = ps;
                        const double pd = double(ps);
                        th[0] = fma(pd, a.winv ? pd * a.winv[j] : pd, th[0]);
                        a.x[j] = a.x[j] + pd;
                    }
                    cta_sum<1>(th);
                }
                if (threadIdx.x == 0) p_th[bid] = th[0];
                if (!coop_barrier(bar, &sh_ok)) return;
                const double theta = coop_total(p_th, 1, 0);
                if (threadIdx.x == 0) upd_done(st, theta);
            }
            __syncthreads();
            ph = st->phase;
        }
        if (ph == PH_SETUP || ph == PH_RUN) {
            const bool init = ph == PH_SETUP;
            double v[2] = {0.0, 0.0};
            for (int32_t sl = __ldg(rwr + w); sl < __ldg(rwr + w + 1); ++sl) {
                const int32_t off = __ldg(a.rsl.ptr + sl);
                const int32_t width = (__ldg(a.rsl.ptr + sl + 1) - off) >> 5;
                row_slot<S>(al, __ldg(a.rsl.seg + 32 * sl + lane), off, width, lane, init, v[0], v[1]);
            }
            cta_sum<2>(v);
            if (threadIdx.x == 0) {
                p_rho[2 * bid] = v[0];
                p_rho[2 * bid + 1] = v[1];
            }
            if (!coop_barrier(bar, &sh_ok)) return;
            const double rho = coop_total(p_rho, 2, 0);
            const double bb = coop_total(p_rho, 2, 1);
            if (threadIdx.x == 0) row_decide(al, st, init, rho, bb);
        }
    }
    __syncthreads();
    if (bid == 0 && threadIdx.x == 0) a.st[0] = sst;
}

// ---------------------------------------------------------------------------
// Auxiliary kernels: products in double, residual norms, column weights
// ---------------------------------------------------------------------------

template <int G, typename S>
__device__ __forceinline__ void spmv_segments(const int32_t *ptr, const int32_t *idx, const S *val,
                                              const Tile &t, const double *v, double *out) {
    for_segments<G>(ptr, t, [&](int32_t seg, int32_t s, int32_t e, int gl, bool valid) {
        const double d = seg_dot<G, S, double, double>(idx, val, s, e, gl, v);
        if (valid && gl == 0) out[seg] = d;
    });
}

// out[seg] = sum over the segment of val * v[idx] (double); with b given,
// part[tile] = sum over the tile of (b - out)^2 (residual norms).
template <typename S>
__global__ void __launch_bounds__(kThreads)
k_spmv(const int32_t *ptr, const int32_t *idx, const void *val_, const Tile *tiles, int32_t ntiles,
       const double *v, double *out, const double *b, double *part) {
    const S *val = static_cast<const S *>(val_);
    for (int32_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tiles[ti];
        switch (t.group & kGroupMask) {
            case 0: {
                const int32_t s = ptr[t.begin], e = ptr[t.begin + 1];
                const double d = cta_dot<S, double, double>(idx, val, s, e, v);
                if (threadIdx.x == 0) out[t.begin] = d;
                break;
            }
            case 1: spmv_segments<1, S>(ptr, idx, val, t, v, out); break;
            case 2: spmv_segments<2, S>(ptr, idx, val, t, v, out); break;
            case 4: spmv_segments<4, S>(ptr, idx, val, t, v, out); break;
            case 8: spmv_segments<8, S>(ptr, idx, val, t, v, out); break;
            case 16: spmv_segments<16, S>(ptr, idx, val, t, v, out); break;
            default: spmv_segments<32, S>(ptr, idx, val, t, v, out); break;
        }
        __syncthreads();
        if (b != nullptr) {
            double acc[1] = {0.0};
            for (int32_t i = t.begin + threadIdx.x; i < t.end; i += kThreads) {
                const double ri = b[i] - out[i];
                acc[0] = fma(ri, ri, acc[0]);
            }
            cta_sum<1>(acc);
            if (threadIdx.x == 0) part[ti] = acc[0];
        }
        __syncthreads();
    }
}

// w_j from the squared norm of column j (segments of the CSC, ascending
// rows): mode 1 -> 1/||A_j||, mode 2 -> 1/||A_j||^2, empty column -> 1;
// winv_j = 1/w_j for theta = p^T W^{-1} p.
template <typename S>
__global__ void k_colweights(const int32_t *ptr, const void *val_, int64_t n, int32_t mode, double *w,
                             double *winv, float *wf, float *winvf) {
    const S *val = static_cast<const S *>(val_);
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n;
         j += int64_t(gridDim.x) * blockDim.x) {
        double ss = 0.0;
        for (int32_t k = ptr[j]; k < ptr[j + 1]; ++k) {
            const double v = double(val[k]);
            ss = __dadd_rn(ss, __dmul_rn(v, v));
        }
        double wj = 1.0, wi = 1.0;
        if (ss != 0.0) {
            const double nrm = __dsqrt_rn(ss);
            wj = mode == 2 ? __ddiv_rn(1.0, ss) : __ddiv_rn(1.0, nrm);
            wi = mode == 2 ? ss : nrm;
        }
        w[j] = wj;
        winv[j] = wi;
        if (wf) {
            wf[j] = float(wj);
            winvf[j] = float(wi);
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

int sweep_ctas_per_sm(int which, bool f32) {
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (which) {
        case 0: e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_row_sweep<float>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_row_sweep<double>, kThreads, 0);
                break;
        case 1: e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_col_sweep<float>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_col_sweep<double>, kThreads, 0);
                break;
        case 3: e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_row_sweep_w<float>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_row_sweep_w<double>, kThreads, 0);
                break;
        case 4: e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_col_sweep_w<float>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_col_sweep_w<double>, kThreads, 0);
                break;
        default: e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update<float>, kThreads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update<double>, kThreads, 0);
                break;
    }
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    // the sweeps over warp ranges run best at four CTAs per SM: more
    // resident warps only add to the L1 requests the random gathers queue
    // behind (C2, FP32 storage: 85.4 us per update at four against 88.4 at
    // the six and eight their registers allow; FP64 column sweep: 40.5 us
    // against 42.0 at six)
    if (which == 3 || which == 4) n = std::min(n, kWarpSweepCtas);
    return n;
}

cudaError_t launch_row_sweep(const SweepArgs &a, bool f32, int grid, cudaStream_t s) {
    if (a.rsl.wr)
        return f32 ? launch_pdl(k_row_sweep_w<float>, grid, s, a) : launch_pdl(k_row_sweep_w<double>, grid, s, a);
    return f32 ? launch_pdl(k_row_sweep<float>, grid, s, a) : launch_pdl(k_row_sweep<double>, grid, s, a);
}

cudaError_t launch_col_sweep(const SweepArgs &a, bool f32, int grid, cudaStream_t s) {
    if (a.csl.wr)
        return f32 ? launch_pdl(k_col_sweep_w<float>, grid, s, a) : launch_pdl(k_col_sweep_w<double>, grid, s, a);
    return f32 ? launch_pdl(k_col_sweep<float>, grid, s, a) : launch_pdl(k_col_sweep<double>, grid, s, a);
}

cudaError_t launch_update(const SweepArgs &a, bool f32, int grid, cudaStream_t s) {
    return f32 ? launch_pdl(k_update<float>, grid, s, a) : launch_pdl(k_update<double>, grid, s, a);
}

cudaError_t launch_cluster_solve(const SweepArgs &a, bool f32, int32_t nsys, int32_t bodies, int32_t vec_bytes,
                                 cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(nsys) * kClusterCtas);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = size_t(vec_bytes > 0 ? vec_bytes : 0);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (vec_bytes <= 0)
        return f32 ? cudaLaunchKernelEx(&cfg, k_cluster_solve<float, false>, a, bodies)
                   : cudaLaunchKernelEx(&cfg, k_cluster_solve<double, false>, a, bodies);
    cudaError_t e = f32 ? cudaFuncSetAttribute(k_cluster_solve<float, true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, vec_bytes)
                        : cudaFuncSetAttribute(k_cluster_solve<double, true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, vec_bytes);
    if (e != cudaSuccess) return e;
    return f32 ? cudaLaunchKernelEx(&cfg, k_cluster_solve<float, true>, a, bodies)
               : cudaLaunchKernelEx(&cfg, k_cluster_solve<double, true>, a, bodies);
}

int coop_ctas_per_sm(bool f32) {
    int n = 0;
    const cudaError_t e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_coop_solve<float>, kThreads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_coop_solve<double>, kThreads, 0);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_coop_solve(const SweepArgs &a, bool f32, int grid, const int32_t *rwr, const int32_t *cwr,
                              double *part, uint32_t *bar, int32_t bodies, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    SweepArgs aa = a;
    void *args[] = {&aa, &rwr, &cwr, &part, &bar, &bodies};
    void *fn = f32 ? reinterpret_cast<void *>(k_coop_solve<float>) : reinterpret_cast<void *>(k_coop_solve<double>);
    return cudaLaunchCooperativeKernel(fn, dim3(unsigned(grid)), dim3(kThreads), args, 0, s);
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
                              double *w, double *winv, float *wf, float *winvf, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int grid = int((n + kThreads - 1) / kThreads);
    if (f32) k_colweights<float><<<grid, kThreads, 0, s>>>(ptr, val, n, mode, w, winv, wf, winvf);
    else k_colweights<double><<<grid, kThreads, 0, s>>>(ptr, val, n, mode, w, winv, wf, winvf);
    return cudaGetLastError();
}

}  // namespace plss
