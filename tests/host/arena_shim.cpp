// Test shim over the serving arena's placement (plss_arena.h): builds with
// g++ alone (no CUDA) so that its invariants are checked on the CPU. Test
// infrastructure only; not part of the library.
#include <cstdint>

#include "plss_arena.h"

using namespace plss;

namespace {
ArenaNeed need_of(const int64_t *q) {
    ArenaNeed n;
    n.m = q[0];
    n.n = q[1];
    n.nnz = q[2];
    n.nsl = q[3];
    n.nel = q[4];
    n.tr = q[5];
    n.tc = q[6];
    n.tv = q[7];
    return n;
}
ArenaPlace place_of(const int64_t *p) {
    ArenaPlace a;
    a.slot = int32_t(p[0]);
    a.roff = p[1];
    a.coff = p[2];
    a.zoff = p[3];
    a.sloff = p[4];
    a.eloff = p[5];
    return a;
}
RangeAlloc &pick(Arena *a, int32_t which) {
    switch (which) {
        case 0: return a->rows;
        case 1: return a->cols;
        case 2: return a->nnzs;
        case 3: return a->slcs;
        default: return a->els;
    }
}
}  // namespace

extern "C" {

void *arena_new(int32_t slots, int64_t mcap, int64_t ncap, int64_t zcap, int64_t slcap, int64_t elcap, int64_t tr,
                int64_t tc, int64_t tv) {
    Arena *a = new Arena();
    a->init(slots, mcap, ncap, zcap, slcap, elcap, tr, tc, tv);
    return a;
}

void arena_free(void *h) { delete static_cast<Arena *>(h); }

// need[8] = m, n, nnz, nsl, nel, tr, tc, tv; out[6] = slot, roff, coff, zoff, sloff, eloff
int32_t arena_place(void *h, const int64_t *need, int64_t *out) {
    ArenaPlace p;
    if (!static_cast<Arena *>(h)->place(need_of(need), p)) return 0;
    out[0] = p.slot;
    out[1] = p.roff;
    out[2] = p.coff;
    out[3] = p.zoff;
    out[4] = p.sloff;
    out[5] = p.eloff;
    return 1;
}

void arena_release(void *h, const int64_t *need, const int64_t *place) {
    static_cast<Arena *>(h)->release(need_of(need), place_of(place));
}

int32_t arena_ever_fits(void *h, const int64_t *need) { return static_cast<Arena *>(h)->ever_fits(need_of(need)); }

// out[0..2] tiles r/c/v, out[3..7] used of rows, cols, nnzs, slcs, els, out[8] taken slots
void arena_counters(void *h, int64_t *out) {
    Arena *a = static_cast<Arena *>(h);
    out[0] = a->tiles_r;
    out[1] = a->tiles_c;
    out[2] = a->tiles_v;
    for (int32_t w = 0; w < 5; ++w) out[3 + w] = pick(a, w).used;
    int64_t t = 0;
    for (uint8_t v : a->taken) t += v;
    out[8] = t;
}

// Free ranges of allocator `which` as (offset, length) pairs; returns their number.
int64_t arena_free_ranges(void *h, int32_t which, int64_t *out, int64_t cap) {
    const RangeAlloc &r = pick(static_cast<Arena *>(h), which);
    int64_t k = 0;
    for (const auto &kv : r.free_) {
        if (k < cap) {
            out[2 * k] = kv.first;
            out[2 * k + 1] = kv.second;
        }
        ++k;
    }
    return k;
}
}
