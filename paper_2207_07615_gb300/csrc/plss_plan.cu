// plss_plan.cu -- the host-side plan of the sweeps: tiles, sliced copies and
// warp ranges. Plain C++ (no CUDA calls), so the same code also builds for
// CPU-only tests of its invariants.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "plss_plan.h"

namespace plss {

// Lanes per segment. FP64 sweeps are bound by the FP64 pipe on GB300, so
// each lane should accumulate about 8 nonzeros (one FMA each, short
// shuffle tree): the largest power of two <= mean/8. FP32 sweeps have FP32
// arithmetic to spare and sum staged products from shared memory: the
// largest power of two <= mean/4. Both within [1, 32].
static int32_t pick_group(double mean, bool f32) {
    const double per_lane = f32 ? 4.0 : 8.0;
    int32_t g = 1;
    while (g < 32 && 2.0 * g * per_lane <= mean) g <<= 1;
    return g;
}

// Cuts segments [begin, end) (offsets in ptr) of system `sys` into tiles of
// about `target` nonzeros; a segment longer than `target` gets a tile of its
// own worked by the whole CTA (group 0). An empty range still gets one
// (empty) tile so that every system reaches its scalar step.
void build_tiles(const int32_t *ptr, int64_t begin, int64_t end, int32_t sys, int64_t target,
                 int64_t max_segs, bool f32, std::vector<Tile> &out) {
    if (begin == end) {
        out.push_back({sys, int32_t(begin), int32_t(begin), 1});
        return;
    }
    int64_t i = begin;
    while (i < end) {
        const int64_t li = int64_t(ptr[i + 1]) - ptr[i];
        if (li > target) {
            out.push_back({sys, int32_t(i), int32_t(i + 1), 0});
            ++i;
            continue;
        }
        int64_t j = i, nz = 0;
        while (j < end && j - i < max_segs) {
            const int64_t l = int64_t(ptr[j + 1]) - ptr[j];
            if (l > target) break;
            if (nz + l > target && j > i) break;
            nz += l;
            ++j;
        }
        // FP32 tiles (cut to the staging limits) stage their products
        out.push_back({sys, int32_t(i), int32_t(j), pick_group(double(nz) / double(j - i), f32) | (f32 ? kStaged : 0)});
        i = j;
    }
}

// Nonzeros per sweep tile for a context of nnz nonzeros: about two tiles
// per resident CTA (a balanced contiguous split), within [1,024, 16,384]
// (2,048 for FP32 storage); then scaled by 2^shift within [256, cap].
int64_t tile_target(int64_t nnz, int64_t slots, bool f32, int32_t shift) {
    // FP32 tiles are staged in 8 KB of shared memory (2,048 float products)
    const int64_t cap = f32 ? 2048 : 16384;
    int64_t t = std::min<int64_t>(cap, std::max<int64_t>(1024, (nnz + 2 * slots - 1) / (2 * slots) * 21 / 20));
    t = shift >= 0 ? t << shift : t >> -shift;
    return std::min<int64_t>(cap, std::max<int64_t>(256, t));
}

// Order of a tile's segments in its slices (decreasing length, ties by
// index); returns the padded element count (32 x each slice's width) for
// slices of 32 / g segments with g lanes each.
static int64_t slice_order(const int32_t *ptr, const Tile &t, std::vector<int32_t> &order, int32_t g) {
    const int32_t nseg = t.end - t.begin, per = 32 / g;
    order.resize(size_t(nseg));
    for (int32_t i = 0; i < nseg; ++i) order[size_t(i)] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return ptr[t.begin + a + 1] - ptr[t.begin + a] > ptr[t.begin + b + 1] - ptr[t.begin + b];
    });
    int64_t padded = 0;
    for (int32_t s = 0; s < nseg; s += per) {
        const int32_t lead = t.begin + order[size_t(s)];
        padded += 32 * int64_t((ptr[lead + 1] - ptr[lead] + g - 1) / g);
    }
    return padded;
}

// Lanes per segment of a side's slices: the largest power of two g with
// 8 g <= mean segment length (at most 32), so that a lane keeps about 8
// elements and wide sides (C2 columns: 40 per column) give every warp
// several slices.
int32_t slice_lanes(int64_t nnz, int64_t segs) {
    int32_t g = 1;
    while (g < 32 && 16 * g * segs <= nnz) g <<= 1;
    return g;
}

// As build_tiles (FP64 sizes), but a tile ends on a multiple of 32
// segments unless a long segment or the end of the range comes first, so
// that only its last slice can be partly empty.
static void cut_slice_tiles(const int32_t *ptr, int64_t begin, int64_t end, int32_t sys, int64_t target,
                            std::vector<Tile> &out) {
    int64_t i = begin;
    while (i < end) {
        if (int64_t(ptr[i + 1]) - ptr[i] > target) {
            out.push_back({sys, int32_t(i), int32_t(i + 1), 0});
            ++i;
            continue;
        }
        int64_t j = i, nz = 0;
        while (j < end && j - i < kTileMaxSegs) {
            int64_t k = j, gz = 0;
            bool stop = false;
            for (; k < end && k < j + 32; ++k) {
                const int64_t l = int64_t(ptr[k + 1]) - ptr[k];
                if (l > target) {
                    stop = true;
                    break;
                }
                gz += l;
            }
            if (k == j || (nz > 0 && nz + gz > target)) break;
            nz += gz;
            j = k;
            if (stop) break;
        }
        out.push_back({sys, int32_t(i), int32_t(j), pick_group(double(nz) / double(j - i), false)});
        i = j;
    }
}

// Tiles of segments [begin, end) of system `sys` for one side of A. With
// `slice`, tiles are cut at the FP64 size on 32-segment boundaries first; a
// tile of short segments whose slices pad it by at most 1/4 is flagged
// kSliced, and the others are cut as they would be without slicing.
void build_side(const int32_t *ptr, int64_t begin, int64_t end, int32_t sys, int64_t nnz, const PlanSlots &slots,
                bool f32, bool slice, int32_t g, std::vector<Tile> &out) {
    const int64_t target = tile_target(nnz, f32 ? slots.f32 : slots.f64, f32, slots.shift);
    if (!slice || begin == end) {
        build_tiles(ptr, begin, end, sys, target, max_segs(f32), f32, out);
        return;
    }
    std::vector<Tile> big;
    cut_slice_tiles(ptr, begin, end, sys, tile_target(nnz, slots.f64, false, slots.shift), big);
    std::vector<int32_t> order;
    for (const Tile &t : big) {
        const int64_t nz = int64_t(ptr[t.end]) - ptr[t.begin];
        if (t.group != 0 && t.end > t.begin && slice_order(ptr, t, order, g) * 4 <= nz * 5) {
            out.push_back({t.sys, t.begin, t.end, t.group | kSliced});
        } else if (t.group != 0 && t.end > t.begin) {
            // uneven segments: staged tiles (FP64 too), so that a long
            // segment does not hold a warp through a serial gather chain
            build_tiles(ptr, t.begin, t.end, sys, f32 ? target : tile_target(nnz, slots.f32, true, slots.shift),
                        max_segs(true), true, out);
        } else {
            out.push_back(t);
        }
    }
}

// The sliced copy of the tiles flagged kSliced (values from v64 or v32),
// g lanes per segment: element k of the segment in slot group q of a slice
// lies in lane q g + (k mod g), row k / g.
void fill_sliced(const int32_t *ptr, const int32_t *idx, const double *v64, const float *v32,
                 const std::vector<Tile> &tiles, int32_t g, HostSliced &out) {
    out = HostSliced();
    out.g = g;
    out.first.resize(tiles.size());
    out.ptr.push_back(0);
    std::vector<int32_t> order;
    const int32_t per = 32 / g;
    for (size_t ti = 0; ti < tiles.size(); ++ti) {
        const Tile &t = tiles[ti];
        out.first[ti] = int32_t(out.ptr.size()) - 1;
        if (!(t.group & kSliced)) continue;
        slice_order(ptr, t, order, g);
        const int32_t nseg = t.end - t.begin;
        for (int32_t s = 0; s < nseg; s += per) {
            const int32_t lead = t.begin + order[size_t(s)];
            const int32_t width = (ptr[lead + 1] - ptr[lead] + g - 1) / g;
            const int32_t base = out.ptr.back();
            out.ptr.push_back(base + 32 * width);
            out.idx.resize(size_t(base) + 32 * size_t(width), -1);
            if (v64) out.v64.resize(out.idx.size(), 0.0);
            else out.v32.resize(out.idx.size(), 0.0f);
            for (int32_t l = 0; l < 32; ++l) {
                const int32_t q = l / g, r = l % g;
                const int32_t seg = s + q < nseg ? t.begin + order[size_t(s + q)] : -1;
                out.seg.push_back(seg);
                if (seg < 0) continue;
                for (int32_t k = r; k < ptr[seg + 1] - ptr[seg]; k += g) {
                    const size_t dst = size_t(base) + 32 * size_t(k / g) + size_t(l);
                    const size_t src = size_t(ptr[seg]) + size_t(k);
                    out.idx[dst] = idx[src];
                    if (v64) out.v64[dst] = v64[src];
                    else out.v32[dst] = v32[src];
                }
            }
        }
    }
}

void build_vec_tiles(int64_t begin, int64_t end, int32_t sys, int64_t chunk, std::vector<Tile> &out) {
    if (begin == end) {
        out.push_back({sys, int32_t(begin), int32_t(begin), 1});
        return;
    }
    for (int64_t i = begin; i < end; i += chunk)
        out.push_back({sys, int32_t(i), int32_t(std::min(end, i + chunk)), 1});
}

// Splits the slices (element offsets sptr) into nwarps contiguous ranges of
// about equal cost: nwarps + 1 boundaries, or nothing unless every tile is
// sliced.
std::vector<int32_t> warp_ranges(const std::vector<Tile> &tiles, const std::vector<int32_t> &sptr, int64_t nwarps) {
    if (tiles.empty() || sptr.size() < 2 || nwarps < 1) return {};
    for (const Tile &t : tiles)
        if (!(t.group & kSliced)) return {};
    // cost of a slice: its elements plus a fixed part (offsets, slot map,
    // results) worth kSliceFixed elements, so that runs of empty slices
    // (empty rows or columns, sorted last) are spread over the warps too
    constexpr int64_t kSliceFixed = 256;
    const int64_t ns = int64_t(sptr.size()) - 1;
    const int64_t total = sptr.back() + kSliceFixed * ns;
    std::vector<int32_t> wr(size_t(nwarps + 1));
    int64_t s = 0;
    for (int64_t w = 0; w < nwarps; ++w) {
        const int64_t goal = total * w / nwarps;   // cost before warp w's first slice
        while (s < ns && sptr[size_t(s)] + kSliceFixed * s < goal) ++s;
        wr[size_t(w)] = int32_t(s);
    }
    wr[size_t(nwarps)] = int32_t(ns);
    return wr;
}

}  // namespace plss
