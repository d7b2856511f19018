// plss_noalloc.cu -- residual r = b - A x and ||r||^2 for callers that cannot
// allocate device memory.
//
// Some callers of this library must not allocate GPU memory once they are
// running: a framework that has handed every byte of the device to its own
// pool (a cudaMalloc from a library would fail or fragment it), or a
// latency-critical loop whose memory is fixed at start-up. For them this file
// offers one entry point that allocates nothing: a row-group kernel of its
// own (8 lanes per row, blocks of 1,024 rows) that forms the same quantity
// as plss_spmv's product followed by b - A x, with its own summation order,
// so the two agree to rounding, not bit for bit. Its scratch -- one partial
// sum per block, an arrival counter and a flag for an invalid CSR -- is one
// file-scope static device array of fixed size instead of context memory.
// Every GPU that loads the library holds that array (about 33 KB) until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "plss.h"
#include "plss_ctx.h"

namespace plss {

constexpr int kNaThreads = 256;
constexpr int kNaLanes = 8;                        // lanes per row
constexpr int64_t kNaRowsPerBlock = 1024;
constexpr int kNaMaxBlocks = 4096;
constexpr int64_t kNaMaxRows = kNaRowsPerBlock * kNaMaxBlocks;   // 4,194,304
constexpr int kNaMaxDevices = 64;

struct NaScratch {
    double part[kNaMaxBlocks];   // one partial sum of r_i^2 per block of 1,024 rows
    unsigned int arrivals;       // blocks finished in the current call
    unsigned int bad;            // set when the CSR broke its contract in this call
};

// The scratch. Host code must not pass &g_na_scratch to a kernel: on the
// host that name is a stand-in, not a device address. The device address is
// fetched once per device with cudaGetSymbolAddress.
static __device__ __align__(256) NaScratch g_na_scratch;

__global__ void __launch_bounds__(kNaThreads)
k_residual_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                   const int32_t *__restrict__ col_idx,
                   const double *__restrict__ val, const double *__restrict__ x,
                   const double *__restrict__ b, double *__restrict__ r, double *norm2,
                   NaScratch *scr) {
    __shared__ double sh[kNaThreads / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = threadIdx.x / kNaLanes, gl = threadIdx.x % kNaLanes;
    const int64_t row0 = int64_t(blockIdx.x) * kNaRowsPerBlock;
    const int64_t row1 = row0 + kNaRowsPerBlock < m ? row0 + kNaRowsPerBlock : m;
    double acc = 0.0;
    bool bad = false;
    // warp-uniform loop: each pass covers kNaThreads / kNaLanes rows. The CSR
    // is not validated on the host (that would need a copy of it), so every
    // access is guarded here: a row range outside [0, nnz] is skipped and a
    // column outside [0, n) is not gathered; either marks the call invalid.
    for (int64_t base = row0; base < row1; base += kNaThreads / kNaLanes) {
        const int64_t row = base + grp;
        const bool ok = row < row1;
        double d = 0.0;
        if (ok) {
            int64_t s = row_ptr[row], e = row_ptr[row + 1];
            if (s < 0 || e > nnz || s > e) {
                bad = true;
                s = e = 0;
            }
            for (int64_t k = s + gl; k < e; k += kNaLanes) {
                const int64_t c = col_idx[k];
                if (c < 0 || c >= n) {
                    bad = true;
                    continue;
                }
                d = fma(val[k], x[c], d);
            }
        }
#pragma unroll
        for (int o = kNaLanes / 2; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (ok && gl == 0) {
            const double ri = b[row] - d;
            r[row] = ri;
            acc += ri * ri;
        }
    }
    if (bad) {
        atomicOr(&scr->bad, 1u);
        __threadfence();
    }
    // fixed-order block sum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) s += sh[w];
        scr->part[blockIdx.x] = s;
        __threadfence();
        s_last = atomicAdd(&scr->arrivals, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += kNaThreads) t += __ldcg(&scr->part[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __syncthreads();
    if (lane == 0) sh[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) s += sh[w];
        *norm2 = __ldcg(&scr->bad) ? __longlong_as_double(0x7ff8000000000000ll) : s;   // NaN: invalid CSR
        scr->arrivals = 0;
        scr->bad = 0;
    }
}

static std::mutex g_na_mu;
static NaScratch *g_na_addr[kNaMaxDevices] = {};

// Device (or managed) memory that the current device `dev` can load from
// with plain loads: device memory must belong to `dev` itself (another
// GPU's buffer would need peer access).
static bool is_device_ptr(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    return at.type == cudaMemoryTypeManaged;
}

}  // namespace plss

using namespace plss;

extern "C" plss_status plss_residual_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                                             const int32_t *col_idx, const double *val, const double *x,
                                             const double *b, double *r, double *norm2, void *stream) {
    clear_error();
    if (m < 0 || n < 0 || nnz < 0) return fail(PLSS_ERR_INVALID, "negative size");
    if (m > kNaMaxRows)
        return fail(PLSS_ERR_INVALID, "m = %lld exceeds the %lld rows the static scratch of "
                    "plss_residual_noalloc covers", (long long)m, (long long)kNaMaxRows);
    if (!row_ptr || !norm2 || (m > 0 && (!b || !r)) || (nnz > 0 && (!col_idx || !val || !x)))
        return fail(PLSS_ERR_INVALID, "NULL array");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        cudaGetLastError();
        return fail(PLSS_ERR_CUDA, "no usable current device");
    }
    const void *rp = row_ptr;
    const void *ptrs[] = {rp, norm2, m > 0 ? static_cast<const void *>(b) : rp,
                          m > 0 ? static_cast<const void *>(r) : rp,
                          nnz > 0 ? static_cast<const void *>(col_idx) : rp,
                          nnz > 0 ? static_cast<const void *>(val) : rp,
                          nnz > 0 ? static_cast<const void *>(x) : rp};
    for (const void *p : ptrs)
        if (!is_device_ptr(p, dev))
            return fail(PLSS_ERR_INVALID, "every array must be device memory of the current device");
    NaScratch *scr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_addr[dev]) {
            // first call on this device: the scratch's device address (in the
            // device's primary context, which the runtime uses; a
            // cudaDeviceReset makes this cached address stale)
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(PLSS_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            }
            g_na_addr[dev] = static_cast<NaScratch *>(p);
        }
        scr = g_na_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(&scr->arrivals, 0, 2 * sizeof(unsigned int), s);   // arrivals, bad
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PLSS_ERR_CUDA, "clearing the scratch counter: %s", cudaGetErrorString(e));
    }
    const int64_t blocks = m > 0 ? (m + kNaRowsPerBlock - 1) / kNaRowsPerBlock : 1;
    k_residual_noalloc<<<unsigned(blocks), kNaThreads, 0, s>>>(m, n, nnz, row_ptr, col_idx, val, x, b, r, norm2,
                                                                scr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PLSS_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return PLSS_OK;
}
