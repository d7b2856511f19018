// plss_arena.h -- where the serving loop puts a system in its device arena:
// first-fit range allocators over the arena's rows, columns, nonzeros and
// sliced slots/elements, and the budgets of slots and tiles. Plain C++ (no
// CUDA), so that the same code also builds for CPU tests of its invariants.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace plss {

// First-fit allocator of integer ranges of [0, cap); a released range merges
// with free neighbours, so releasing everything leaves one free range.
struct RangeAlloc {
    int64_t cap = 0, used = 0;
    std::map<int64_t, int64_t> free_;   // offset -> length of each free range
    void init(int64_t c) {
        cap = c;
        used = 0;
        free_.clear();
        if (c > 0) free_[0] = c;
    }
    // The lowest free range of at least len entries; len <= 0 takes nothing
    // (offset 0).
    bool alloc(int64_t len, int64_t &off) {
        off = 0;
        if (len <= 0) return true;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                off = it->first;
                const int64_t rest = it->second - len;
                free_.erase(it);
                if (rest) free_[off + len] = rest;
                used += len;
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t len) {
        if (len <= 0) return;
        used -= len;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// What one system takes: m + 1 row entries (row pointer), n + 1 column
// entries, nnz nonzeros, slice slots and sliced elements (0 without sliced
// copies), and row / column / vector tiles.
struct ArenaNeed {
    int64_t m = 0, n = 0, nnz = 0, nsl = 0, nel = 0;
    int64_t tr = 0, tc = 0, tv = 0;
};

// Where a placed system lives.
struct ArenaPlace {
    int32_t slot = -1;
    int64_t roff = 0, coff = 0, zoff = 0, sloff = 0, eloff = 0;
};

struct Arena {
    RangeAlloc rows, cols, nnzs, slcs, els;
    int64_t Tr = 0, Tc = 0, Tv = 0;                  // tile budgets
    int64_t tiles_r = 0, tiles_c = 0, tiles_v = 0;   // tiles of the placed systems
    std::vector<uint8_t> taken;                      // per slot

    void init(int32_t slots, int64_t mcap, int64_t ncap, int64_t zcap, int64_t slcap, int64_t elcap, int64_t tr,
              int64_t tc, int64_t tv) {
        rows.init(mcap);
        cols.init(ncap);
        nnzs.init(zcap);
        slcs.init(slcap);
        els.init(elcap);
        Tr = tr;
        Tc = tc;
        Tv = tv;
        tiles_r = tiles_c = tiles_v = 0;
        taken.assign(size_t(slots > 0 ? slots : 0), 0);
    }

    // Whether a system could be placed in the empty arena.
    bool ever_fits(const ArenaNeed &q) const {
        return !taken.empty() && q.m + 1 <= rows.cap && q.n + 1 <= cols.cap && q.nnz <= nnzs.cap &&
               q.nsl <= slcs.cap && q.nel <= els.cap && q.tr <= Tr && q.tc <= Tc && q.tv <= Tv;
    }

    // Places a system all or nothing: the lowest free slot, the tile budgets,
    // then first-fit ranges; on failure nothing has changed.
    bool place(const ArenaNeed &q, ArenaPlace &p) {
        int32_t slot = -1;
        for (size_t i = 0; i < taken.size(); ++i)
            if (!taken[i]) {
                slot = int32_t(i);
                break;
            }
        if (slot < 0) return false;
        if (tiles_r + q.tr > Tr || tiles_c + q.tc > Tc || tiles_v + q.tv > Tv) return false;
        ArenaPlace at;
        at.slot = slot;
        if (!rows.alloc(q.m + 1, at.roff)) return false;
        if (!cols.alloc(q.n + 1, at.coff)) {
            rows.release(at.roff, q.m + 1);
            return false;
        }
        if (!nnzs.alloc(q.nnz, at.zoff)) {
            rows.release(at.roff, q.m + 1);
            cols.release(at.coff, q.n + 1);
            return false;
        }
        if (!slcs.alloc(q.nsl, at.sloff)) {
            rows.release(at.roff, q.m + 1);
            cols.release(at.coff, q.n + 1);
            nnzs.release(at.zoff, q.nnz);
            return false;
        }
        if (!els.alloc(q.nel, at.eloff)) {
            rows.release(at.roff, q.m + 1);
            cols.release(at.coff, q.n + 1);
            nnzs.release(at.zoff, q.nnz);
            slcs.release(at.sloff, q.nsl);
            return false;
        }
        taken[size_t(slot)] = 1;
        tiles_r += q.tr;
        tiles_c += q.tc;
        tiles_v += q.tv;
        p = at;
        return true;
    }

    // Gives back what place() took for (q, p).
    void release(const ArenaNeed &q, const ArenaPlace &p) {
        rows.release(p.roff, q.m + 1);
        cols.release(p.coff, q.n + 1);
        nnzs.release(p.zoff, q.nnz);
        slcs.release(p.sloff, q.nsl);
        els.release(p.eloff, q.nel);
        tiles_r -= q.tr;
        tiles_c -= q.tc;
        tiles_v -= q.tv;
        if (p.slot >= 0 && size_t(p.slot) < taken.size()) taken[size_t(p.slot)] = 0;
    }
};

}  // namespace plss
