// Test shim over the host-side plan of the sweeps (plss_plan.cu): builds
// with g++ alone (no CUDA) so the plan's invariants are checked on the CPU.
// Test infrastructure only; not part of the library.
#include <cstdint>
#include <cstring>
#include <vector>

#include "plss_plan.h"

using namespace plss;

namespace {
struct Plan {
    std::vector<Tile> tiles;
    HostSliced sl;
    std::vector<int32_t> wr;
};
}  // namespace

extern "C" {

int32_t shim_slice_lanes(int64_t nnz, int64_t segs) { return slice_lanes(nnz, segs); }

int64_t shim_tile_target(int64_t nnz, int64_t slots, int32_t f32, int32_t shift) {
    return tile_target(nnz, slots, f32 != 0, shift);
}

// One side of a single system: segments [0, nseg) with offsets ptr[nseg+1]
// (int32), indices idx and double values val.
void *shim_plan(const int32_t *ptr, const int32_t *idx, const double *val, int64_t nseg, int64_t nnz,
                int64_t slots64, int64_t slots32, int32_t f32, int32_t slice, int32_t g, int64_t nwarps,
                int32_t shift) {
    Plan *p = new Plan();
    PlanSlots s;
    s.f64 = slots64;
    s.f32 = slots32;
    s.shift = shift;
    build_side(ptr, 0, nseg, 0, nnz, s, f32 != 0, slice != 0, g, p->tiles);
    fill_sliced(ptr, idx, val, nullptr, p->tiles, g, p->sl);
    p->wr = warp_ranges(p->tiles, p->sl.ptr, nwarps);
    return p;
}

// Sizes: 0 tiles (x4 int32), 1 first, 2 ptr, 3 seg, 4 idx (= values), 5 warp ranges.
int64_t shim_count(void *h, int32_t which) {
    const Plan *p = static_cast<const Plan *>(h);
    switch (which) {
        case 0: return int64_t(p->tiles.size());
        case 1: return int64_t(p->sl.first.size());
        case 2: return int64_t(p->sl.ptr.size());
        case 3: return int64_t(p->sl.seg.size());
        case 4: return int64_t(p->sl.idx.size());
        default: return int64_t(p->wr.size());
    }
}

void shim_copy(void *h, int32_t which, void *dst) {
    const Plan *p = static_cast<const Plan *>(h);
    switch (which) {
        case 0: std::memcpy(dst, p->tiles.data(), p->tiles.size() * sizeof(Tile)); break;
        case 1: std::memcpy(dst, p->sl.first.data(), p->sl.first.size() * 4); break;
        case 2: std::memcpy(dst, p->sl.ptr.data(), p->sl.ptr.size() * 4); break;
        case 3: std::memcpy(dst, p->sl.seg.data(), p->sl.seg.size() * 4); break;
        case 4: std::memcpy(dst, p->sl.idx.data(), p->sl.idx.size() * 4); break;
        case 6: std::memcpy(dst, p->sl.v64.data(), p->sl.v64.size() * 8); break;
        default: std::memcpy(dst, p->wr.data(), p->wr.size() * 4); break;
    }
}

void shim_free(void *h) { delete static_cast<Plan *>(h); }
}
