// plss_probe.cu -- the gather bound of a context's sweeps, measured on the
// device.
//
// Every nonzero of a residual-sketch sweep gathers one entry of a dense
// vector at a column (row sweep, A p) or row (column sweep, A^T r) given by
// the matrix, and on GB300 those random gathers, not HBM bytes, set the
// sweeps' time. plss_gather_bound runs a kernel that does only that: it
// walks the same sliced index stream with the same grid and warp ranges as
// the sweep and gathers the same vector, and does nothing else -- no values,
// no products, no row sums, no writes of r or u, no reductions. Its time is
// the floor the sweep's gathers alone would take, so sweep time / this time
// says how much the sweep's own arithmetic and bookkeeping add.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "plss.h"
#include "plss_ctx.h"
#include "plss_dev.cuh"
#include "plss_launch.h"

namespace plss {

__device__ __forceinline__ unsigned long long gbits(double v) {
    return static_cast<unsigned long long>(__double_as_longlong(v));
}
__device__ __forceinline__ unsigned long long gbits(float v) { return __float_as_uint(v); }

// Warp w walks slices [wr[w], wr[w + 1]) of `sl` exactly as the sweep over
// warp ranges does (8 index loads, then their 8 gathers) and folds the
// gathered bits with XOR (integer ALU only); a store guarded by a value the
// compiler cannot know (`magic`, passed at run time and never matched in
// practice) keeps every load alive.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gather_slices(Sliced sl, const T *__restrict__ x,
                                                            unsigned long long magic,
                                                            unsigned long long *sink) {
    const int lane = threadIdx.x & 31;
    const int32_t w = int32_t(threadIdx.x >> 5) * int32_t(gridDim.x) + int32_t(blockIdx.x);   // as the sweeps
    const int32_t s0 = __ldg(sl.wr + w), s1 = __ldg(sl.wr + w + 1);
    unsigned long long acc = 0;
    for (int32_t s = s0; s < s1; ++s) {
        const int32_t off = __ldg(sl.ptr + s);
        const int32_t width = (__ldg(sl.ptr + s + 1) - off) >> 5;
        for (int32_t k0 = 0; k0 < width; k0 += 8) {
            int32_t c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) c[u] = k0 + u < width ? __ldg(sl.idx + off + 32 * (k0 + u) + lane) : -1;
            T g[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) g[u] = c[u] >= 0 ? __ldcg(x + c[u]) : T(0);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc ^= gbits(g[u]);
        }
    }
    if (acc == magic) sink[0] = acc;
}

// Writes `n16` 16-byte words: evicts the gathered vector and the index
// stream from L2 between timed runs.
__global__ void k_flush_l2(int4 *buf, int64_t n16, int v) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += int64_t(gridDim.x) * blockDim.x)
        buf[i] = make_int4(v, v, v, v);
}

// Reads x once, leaving it in L2 as the solve does (the sweep that gathers
// a vector runs right after the kernel that wrote it).
template <typename T>
__global__ void k_touch(const T *__restrict__ x, int64_t n, unsigned long long magic, unsigned long long *sink) {
    unsigned long long a = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a ^= gbits(x[i]);
    if (a == magic) sink[0] = a;
}

}  // namespace plss

using namespace plss;

extern "C" plss_status plss_gather_bound(plss_ctx *c, int32_t side, int32_t reps, double *us_median,
                                         double *us_min) {
    clear_error();
    if (!c) return fail(PLSS_ERR_INVALID, "NULL context");
    if (side != 0 && side != 1) return fail(PLSS_ERR_INVALID, "side must be 0 (rows) or 1 (columns)");
    if (reps < 1 || reps > 1000) return fail(PLSS_ERR_INVALID, "reps must be in [1, 1000]");
    const Sliced &sl = side == 0 ? c->rsl : c->csl;
    const int32_t *wr = side == 0 ? c->d_rwr : c->d_cwr;
    if (c->nsys != 1 || !wr || !sl.idx)
        return fail(PLSS_ERR_INVALID, "the gather bound needs a single-system context whose side is "
                    "sliced throughout (the sweeps then run over warp ranges)");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(PLSS_ERR_CUDA, "cudaSetDevice");
    const int grid = side == 0 ? c->grid_r : c->grid_c;
    const void *x = side == 0 ? c->d_p : c->d_r;
    const int64_t len = side == 0 ? c->n : c->m;
    const int64_t flush_bytes = int64_t(256) << 20;
    void *flush = nullptr, *sink = nullptr;
    plss_status st = dalloc(&flush, size_t(flush_bytes), "L2 flush buffer");
    if (st != PLSS_OK) return st;
    st = dalloc(&sink, sizeof(unsigned long long), "sink");
    if (st != PLSS_OK) {
        dfree(flush);
        return st;
    }
    cudaStream_t s = c->cap_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> t;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    Sliced a = sl;
    a.wr = wr;
    const unsigned long long magic = 0x00000000deadbeefull;   // a 32-bit value: reachable for float too
    for (int32_t i = 0; i < reps + 1 && e == cudaSuccess; ++i) {
        k_flush_l2<<<c->nsm * 4, 256, 0, s>>>(static_cast<int4 *>(flush), flush_bytes / 16, i);
        if (c->f32) {
            k_touch<float><<<c->nsm * 4, 256, 0, s>>>(static_cast<const float *>(x), len, magic,
                                                      static_cast<unsigned long long *>(sink));
        } else {
            k_touch<double><<<c->nsm * 4, 256, 0, s>>>(static_cast<const double *>(x), len, magic,
                                                       static_cast<unsigned long long *>(sink));
        }
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        if (c->f32) {
            k_gather_slices<float><<<grid, kThreads, 0, s>>>(a, static_cast<const float *>(x), magic,
                                                              static_cast<unsigned long long *>(sink));
        } else {
            k_gather_slices<double><<<grid, kThreads, 0, s>>>(a, static_cast<const double *>(x), magic,
                                                               static_cast<unsigned long long *>(sink));
        }
        e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && i > 0) t.push_back(ms);   // the first run warms up
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(flush);
    dfree(sink);
    if (e != cudaSuccess) return fail(PLSS_ERR_CUDA, "gather bound: %s", cudaGetErrorString(e));
    std::sort(t.begin(), t.end());
    if (us_median) *us_median = 1e3 * double(t[t.size() / 2]);
    if (us_min) *us_min = 1e3 * double(t.front());
    return PLSS_OK;
}
