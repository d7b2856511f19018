// plss_launch.h -- host-side launchers of the device kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "plss_dev.cuh"

namespace plss {

// Residual-sketch sweeps (plss_kernels.cu). f32 selects float storage of A
// and of the vectors r, p, u.
cudaError_t launch_row_sweep(const SweepArgs &a, bool f32, int grid, cudaStream_t s);
cudaError_t launch_col_sweep(const SweepArgs &a, bool f32, int grid, cudaStream_t s);
cudaError_t launch_update(const SweepArgs &a, bool f32, int grid, cudaStream_t s);

// Small systems: one cluster of 8 CTAs per system of the context runs up to
// `bodies` bodies of the recursion (column sweep, update, row sweep).
// vec_bytes > 0: every CTA keeps copies of r and p in that many bytes of
// shared memory (at least (m + n) x the storage size of the largest system;
// at most kClusterVecBytes); 0: the vectors are read from global memory.
constexpr int32_t kClusterVecBytes = 128 * 1024;
cudaError_t launch_cluster_solve(const SweepArgs &a, bool f32, int32_t nsys, int32_t bodies, int32_t vec_bytes,
                                 cudaStream_t s);

// One system on the whole GPU (schedule COOP): up to `bodies` bodies per
// cooperative launch of `grid` CTAs (all resident), with this grid's warp
// ranges of the sliced rows and columns, per-CTA partials part[4 * grid]
// and barrier words bar[4] (cleared by the launcher). coop_ctas_per_sm: the
// kernel's resident CTAs per SM (0 when it cannot run).
int coop_ctas_per_sm(bool f32);
cudaError_t launch_coop_solve(const SweepArgs &a, bool f32, int grid, const int32_t *rwr, const int32_t *cwr,
                              double *part, uint32_t *bar, int32_t bodies, cudaStream_t s);

// Resident CTAs per SM of a sweep kernel (0 row, 1 column, 2 update, 3 row
// and 4 column over warp ranges).
int sweep_ctas_per_sm(int which, bool f32);

// out[seg] = (A v)[seg] over the segments of `tiles` in double; with b,
// part[tile] = sum over the tile of (b - out)^2.
cudaError_t launch_spmv(const int32_t *ptr, const int32_t *idx, const void *val, bool f32,
                        const Tile *tiles, int32_t ntiles, const double *v, double *out,
                        const double *b, double *part, int grid, cudaStream_t s);

// Diagonal weights of Sec. 4.1 from column segments (ptr over n columns):
// w[j] and winv[j] = 1/w[j] (and float copies when wf is not null).
cudaError_t launch_colweights(const int32_t *ptr, const void *val, bool f32, int64_t n,
                              int32_t mode, double *w, double *winv, float *wf, float *winvf,
                              cudaStream_t s);


// Launch with the programmatic-stream-serialization attribute (captured as
// programmatic edges in CUDA graphs): the next sweep's launch overlaps the
// tail of the previous one and its CTAs wait in wait_prior_grid().
template <typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Args...), int grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace plss
