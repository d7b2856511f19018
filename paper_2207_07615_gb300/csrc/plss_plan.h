// plss_plan.h -- host-side plan of the sweeps (plss_plan.cu): plain C++.
#pragma once

#include <cstdint>
#include <vector>

#include "plss_dev.cuh"

namespace plss {

constexpr int64_t kTileMaxSegs = 2048;      // max rows/columns per FP64 sweep tile
constexpr int64_t kTileMaxSegsF32 = 1024;   // ... per staged tile (shared-memory staging)
inline int64_t max_segs(bool f32) { return f32 ? kTileMaxSegsF32 : kTileMaxSegs; }

// Resident CTA slots of the sweeps on the device (SMs x CTAs per SM) for
// FP64 and FP32 storage; sizes the tiles. `shift` scales the tiles' target
// nonzeros by 2^shift (the autotuner's knob; 0 = the default plan).
struct PlanSlots {
    int64_t f64 = 1, f32 = 1;
    int32_t shift = 0;
};

// Host copy of a sliced side (layout in plss_dev.cuh).
struct HostSliced {
    int32_t g = 1;   // lanes per segment
    std::vector<int32_t> first, ptr, seg, idx;
    std::vector<double> v64;
    std::vector<float> v32;
};

void build_tiles(const int32_t *ptr, int64_t begin, int64_t end, int32_t sys, int64_t target,
                 int64_t max_segs, bool f32, std::vector<Tile> &out);
int64_t tile_target(int64_t nnz, int64_t slots, bool f32, int32_t shift = 0);
void build_vec_tiles(int64_t begin, int64_t end, int32_t sys, int64_t chunk, std::vector<Tile> &out);
int32_t slice_lanes(int64_t nnz, int64_t segs);
void build_side(const int32_t *ptr, int64_t begin, int64_t end, int32_t sys, int64_t nnz, const PlanSlots &slots,
                bool f32, bool slice, int32_t g, std::vector<Tile> &out);
void fill_sliced(const int32_t *ptr, const int32_t *idx, const double *v64, const float *v32,
                 const std::vector<Tile> &tiles, int32_t g, HostSliced &out);
std::vector<int32_t> warp_ranges(const std::vector<Tile> &tiles, const std::vector<int32_t> &sptr, int64_t nwarps);

}  // namespace plss
