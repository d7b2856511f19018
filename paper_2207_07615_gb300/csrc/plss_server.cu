// plss_server.cu -- continuous-batching PLSS solve server.
//
// One host worker thread owns a device arena (CSR + transpose + vectors of
// every resident system, plus tile schedules and per-system state) and runs
// rounds:  retire finished systems -> admit queued requests into freed slots
// and arena ranges -> rebuild the concatenated tile lists -> run a few
// iterations of Algorithm 1 for all resident systems at once.
// Every sweep is one launch over the tiles of all resident systems; each
// system keeps its own scalars, stopping test and status, so a system's
// arithmetic is the same as when it runs alone (its tiles, partial sums and
// reduction order do not depend on its neighbours).
//
// The host-side work of a request (validation, transpose, tile schedule)
// runs in plss_submit on the caller's thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plss.h"
#include "plss_arena.h"
#include "plss_ctx.h"
#include "plss_dev.cuh"
#include "plss_launch.h"
#include "plss_trace.h"

namespace plss {

struct SrvRequest {
    uint64_t ticket = 0;
    int64_t m = 0, n = 0, nnz = 0;
    // local arrays (0-based), ready to be offset into the arena
    std::vector<int32_t> rp, ci, cp, ri;
    std::vector<double> v64, cv64;
    std::vector<float> v32, cv32;
    std::vector<Tile> rt, ct, vt;   // local segment indices, sys = 0
    HostSliced hr, hc;              // sliced copies of the rows / columns (local indices)
    int64_t nsl = 0, nel = 0;       // slice slots and elements they take in the arena
    std::vector<double> b, x0;
    double tol = 1e-8;
    int64_t maxit = -1;
    int32_t w_mode = 0;
    std::chrono::steady_clock::time_point t_submit;
    // placement
    int32_t slot = -1;
    int64_t roff = 0, coff = 0, zoff = 0, sloff = 0, eloff = 0;
    int32_t rt_begin = 0, ct_begin = 0, vt_begin = 0;
    // outcome
    std::vector<double> x;
    plss_result res{};

    ArenaNeed need() const {
        ArenaNeed q;
        q.m = m;
        q.n = n;
        q.nnz = nnz;
        q.nsl = nsl;
        q.nel = nel;
        q.tr = int64_t(rt.size());
        q.tc = int64_t(ct.size());
        q.tv = int64_t(vt.size());
        return q;
    }
    ArenaPlace place() const {
        ArenaPlace p;
        p.slot = slot;
        p.roff = roff;
        p.coff = coff;
        p.zoff = zoff;
        p.sloff = sloff;
        p.eloff = eloff;
        return p;
    }
};

}  // namespace plss

struct plss_server {
    plss_server_opts so{};
    bool f32 = false;
    int device = 0, nsm = 1;
    int64_t Mcap = 0, Ncap = 0, Zcap = 0, Tr = 0, Tc = 0, Tv = 0;
    int32_t Scap = 0;
    bool sliced = false;                 // PLSS_LAYOUT_AUTO: sliced copies in the arena
    int64_t SLcap = 0, ELcap = 0;        // slice slots, sliced elements
    plss::Arena arena;                   // placement of the resident systems
    int32_t *d_sl_ptr = nullptr, *d_sl_seg = nullptr, *d_sl_idx = nullptr, *d_rfirst = nullptr,
            *d_cfirst = nullptr;
    void *d_sl_val = nullptr;
    int32_t *d_row_ptr = nullptr, *d_col_idx = nullptr, *d_col_ptr = nullptr, *d_row_idx = nullptr;
    void *d_val = nullptr, *d_cval = nullptr, *d_r = nullptr, *d_p = nullptr, *d_u = nullptr;
    double *d_b = nullptr, *d_x = nullptr, *d_w = nullptr, *d_vout = nullptr;
    float *d_wf = nullptr;   // FP32 servers: float w and 1/w
    double *d_part_row = nullptr, *d_part_col = nullptr, *d_part_upd = nullptr, *d_part_res = nullptr;
    plss::Tile *d_rt = nullptr, *d_ct = nullptr, *d_vt = nullptr;
    plss::SysDesc *d_desc = nullptr;
    plss::SysState *d_st = nullptr;
    int32_t *d_active = nullptr;
    plss::SysState *h_st = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<plss::SysDesc> h_desc;
    std::vector<plss::SrvRequest *> slot_req;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<plss::SrvRequest *> queue;
    std::unordered_map<uint64_t, plss::SrvRequest *> done;
    std::unordered_map<uint64_t, int> live;   // ticket -> 1 while queued or running
    uint64_t next_ticket = 1;
    int64_t completed = 0, running = 0;
    int64_t bytes_per_row = 0, bytes_per_col = 0, bytes_per_nnz = 0;
    std::atomic<bool> stop{false};
    std::string fatal;
    std::thread worker;
};

namespace plss {

static size_t sval(const plss_server *s) { return s->f32 ? 4 : 8; }

static void srv_free_device(plss_server *s) {
    void *ptrs[] = {s->d_row_ptr, s->d_col_idx, s->d_col_ptr, s->d_row_idx, s->d_val, s->d_cval,
                    s->d_r, s->d_p, s->d_u, s->d_b, s->d_x, s->d_w, s->d_wf, s->d_vout, s->d_part_row,
                    s->d_part_col, s->d_part_upd, s->d_part_res, s->d_rt, s->d_ct, s->d_vt,
                    s->d_desc, s->d_st, s->d_active, s->d_sl_ptr, s->d_sl_seg, s->d_sl_idx,
                    s->d_sl_val, s->d_rfirst, s->d_cfirst};
    for (void *p : ptrs) dfree(p);
    if (s->h_st) cudaFreeHost(s->h_st);
    if (s->stream) cudaStreamDestroy(s->stream);
}

// Host preparation of a request: local CSR (int32 offsets), transpose,
// tile schedules.
static void srv_prepare(plss_server *s, HostCsr &h, SrvRequest *r) {
    r->m = h.m;
    r->n = h.n;
    r->nnz = h.nnz;
    r->rp.resize(size_t(h.m + 1));
    for (int64_t i = 0; i <= h.m; ++i) r->rp[size_t(i)] = int32_t(h.row_ptr[size_t(i)]);
    r->ci = h.col_idx;
    r->cp.assign(size_t(h.n + 1), 0);
    r->ri.resize(size_t(h.nnz));
    for (int64_t k = 0; k < h.nnz; ++k) r->cp[size_t(r->ci[size_t(k)] + 1)] += 1;
    for (int64_t j = 0; j < h.n; ++j) r->cp[size_t(j + 1)] += r->cp[size_t(j)];
    std::vector<int32_t> next(r->cp.begin(), r->cp.end() - 1);
    std::vector<double> cv(static_cast<size_t>(h.nnz));
    for (int64_t i = 0; i < h.m; ++i)
        for (int32_t k = r->rp[size_t(i)]; k < r->rp[size_t(i + 1)]; ++k) {
            const int32_t dst = next[size_t(r->ci[size_t(k)])]++;
            r->ri[size_t(dst)] = int32_t(i);
            cv[size_t(dst)] = h.val[size_t(k)];
        }
    if (s->f32) {
        r->v32.assign(h.val.begin(), h.val.end());
        r->cv32.assign(cv.begin(), cv.end());
    } else {
        r->v64 = std::move(h.val);
        r->cv64 = std::move(cv);
    }
    // the request's own schedule (it does not depend on its neighbours, so
    // its arithmetic is the same alone and in the mix): as a single-system
    // context would cut it (CSR layout), or with sliced tiles, one lane per
    // segment (AUTO)
    const PlanSlots slots = plan_slots(s->nsm);
    if (s->sliced) {
        build_side(r->rp.data(), 0, h.m, 0, h.nnz, slots, s->f32, true, 1, r->rt);
        build_side(r->cp.data(), 0, h.n, 0, h.nnz, slots, s->f32, true, 1, r->ct);
        const double *v = s->f32 ? nullptr : r->v64.data(), *cvv = s->f32 ? nullptr : r->cv64.data();
        const float *vf = s->f32 ? r->v32.data() : nullptr, *cvf = s->f32 ? r->cv32.data() : nullptr;
        fill_sliced(r->rp.data(), r->ci.data(), v, vf, r->rt, 1, r->hr);
        fill_sliced(r->cp.data(), r->ri.data(), cvv, cvf, r->ct, 1, r->hc);
        r->nsl = int64_t(r->hr.ptr.size() + r->hc.ptr.size());
        r->nel = int64_t(r->hr.idx.size() + r->hc.idx.size());
    } else {
        const int64_t target = tile_target(h.nnz, s->f32 ? slots.f32 : slots.f64, s->f32);
        build_tiles(r->rp.data(), 0, h.m, 0, target, max_segs(s->f32), s->f32, r->rt);
        build_tiles(r->cp.data(), 0, h.n, 0, target, max_segs(s->f32), s->f32, r->ct);
    }
    build_vec_tiles(0, h.n, 0, kVecTile, r->vt);
}

// Arena ranges and a slot for r; false (nothing taken) when they do not fit.
static bool srv_place(plss_server *s, SrvRequest *r) {
    ArenaPlace at;
    if (!s->arena.place(r->need(), at)) return false;
    r->slot = at.slot;
    r->roff = at.roff;
    r->coff = at.coff;
    r->zoff = at.zoff;
    r->sloff = at.sloff;
    r->eloff = at.eloff;
    s->slot_req[size_t(at.slot)] = r;
    return true;
}

static void srv_unplace(plss_server *s, SrvRequest *r) {
    s->arena.release(r->need(), r->place());
    s->slot_req[size_t(r->slot)] = nullptr;
}

#define SRV_TRY(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            s->fatal = std::string(#expr) + ": " + cudaGetErrorString(e_);                 \
            return false;                                                                  \
        }                                                                                  \
    } while (0)

// Copies a placed request into the arena and sets its state to start.
static bool srv_upload(plss_server *s, SrvRequest *r) {
    cudaStream_t st = s->stream;
    const size_t sb = sval(s);
    std::vector<int32_t> rp(r->rp.size()), ci(r->ci.size()), cp(r->cp.size()), ri(r->ri.size());
    for (size_t i = 0; i < rp.size(); ++i) rp[i] = int32_t(r->zoff) + r->rp[i];
    for (size_t k = 0; k < ci.size(); ++k) ci[k] = int32_t(r->coff) + r->ci[k];
    for (size_t j = 0; j < cp.size(); ++j) cp[j] = int32_t(r->zoff) + r->cp[j];
    for (size_t k = 0; k < ri.size(); ++k) ri[k] = int32_t(r->roff) + r->ri[k];
    SRV_TRY(cudaMemcpyAsync(s->d_row_ptr + r->roff, rp.data(), 4 * rp.size(), cudaMemcpyHostToDevice, st));
    SRV_TRY(cudaMemcpyAsync(s->d_col_ptr + r->coff, cp.data(), 4 * cp.size(), cudaMemcpyHostToDevice, st));
    if (r->nnz > 0) {
        SRV_TRY(cudaMemcpyAsync(s->d_col_idx + r->zoff, ci.data(), 4 * ci.size(), cudaMemcpyHostToDevice, st));
        SRV_TRY(cudaMemcpyAsync(s->d_row_idx + r->zoff, ri.data(), 4 * ri.size(), cudaMemcpyHostToDevice, st));
        const void *v = s->f32 ? static_cast<const void *>(r->v32.data()) : static_cast<const void *>(r->v64.data());
        const void *cv = s->f32 ? static_cast<const void *>(r->cv32.data()) : static_cast<const void *>(r->cv64.data());
        SRV_TRY(cudaMemcpyAsync(static_cast<char *>(s->d_val) + sb * size_t(r->zoff), v, sb * size_t(r->nnz),
                                cudaMemcpyHostToDevice, st));
        SRV_TRY(cudaMemcpyAsync(static_cast<char *>(s->d_cval) + sb * size_t(r->zoff), cv, sb * size_t(r->nnz),
                                cudaMemcpyHostToDevice, st));
    }
    if (r->nsl > 0) {
        // the sliced copies with arena offsets: element offsets, segment ids
        // and indices become global; rows' slices first, then columns'
        const HostSliced *side[2] = {&r->hr, &r->hc};
        const int64_t seg_off[2] = {r->roff, r->coff}, idx_off[2] = {r->coff, r->roff};
        int64_t so = r->sloff, eo = r->eloff;
        for (int q = 0; q < 2; ++q) {
            const HostSliced &h = *side[q];
            std::vector<int32_t> ptr(h.ptr.size()), seg(h.seg.size()), idx(h.idx.size());
            for (size_t i = 0; i < ptr.size(); ++i) ptr[i] = int32_t(eo + h.ptr[i]);
            for (size_t i = 0; i < seg.size(); ++i) seg[i] = h.seg[i] < 0 ? -1 : int32_t(seg_off[q] + h.seg[i]);
            for (size_t i = 0; i < idx.size(); ++i) idx[i] = h.idx[i] < 0 ? -1 : int32_t(idx_off[q] + h.idx[i]);
            SRV_TRY(cudaMemcpyAsync(s->d_sl_ptr + so, ptr.data(), 4 * ptr.size(), cudaMemcpyHostToDevice, st));
            if (!seg.empty())
                SRV_TRY(cudaMemcpyAsync(s->d_sl_seg + 32 * so, seg.data(), 4 * seg.size(), cudaMemcpyHostToDevice, st));
            if (!idx.empty()) {
                SRV_TRY(cudaMemcpyAsync(s->d_sl_idx + eo, idx.data(), 4 * idx.size(), cudaMemcpyHostToDevice, st));
                const void *v = s->f32 ? static_cast<const void *>(h.v32.data()) : static_cast<const void *>(h.v64.data());
                SRV_TRY(cudaMemcpyAsync(static_cast<char *>(s->d_sl_val) + sb * size_t(eo), v, sb * idx.size(),
                                        cudaMemcpyHostToDevice, st));
            }
            SRV_TRY(cudaStreamSynchronize(st));   // the host staging vectors go out of scope
            so += int64_t(h.ptr.size());
            eo += int64_t(h.idx.size());
        }
    }
    if (r->m > 0) SRV_TRY(cudaMemcpyAsync(s->d_b + r->roff, r->b.data(), 8 * size_t(r->m), cudaMemcpyHostToDevice, st));
    if (r->n > 0) {
        if (r->x0.empty()) SRV_TRY(cudaMemsetAsync(s->d_x + r->coff, 0, 8 * size_t(r->n), st));
        else SRV_TRY(cudaMemcpyAsync(s->d_x + r->coff, r->x0.data(), 8 * size_t(r->n), cudaMemcpyHostToDevice, st));
        if (r->w_mode == PLSS_W_IDENTITY) {
            std::vector<double> ones(static_cast<size_t>(r->n), 1.0);
            SRV_TRY(cudaMemcpyAsync(s->d_w + r->coff, ones.data(), 8 * size_t(r->n), cudaMemcpyHostToDevice, st));
            SRV_TRY(cudaMemcpyAsync(s->d_w + s->Ncap + r->coff, ones.data(), 8 * size_t(r->n),
                                    cudaMemcpyHostToDevice, st));
            if (s->d_wf) {
                std::vector<float> fones(static_cast<size_t>(2 * r->n), 1.0f);
                SRV_TRY(cudaMemcpyAsync(s->d_wf + r->coff, fones.data(), 4 * size_t(r->n), cudaMemcpyHostToDevice, st));
                SRV_TRY(cudaMemcpyAsync(s->d_wf + s->Ncap + r->coff, fones.data(), 4 * size_t(r->n),
                                        cudaMemcpyHostToDevice, st));
                SRV_TRY(cudaStreamSynchronize(st));
            }
        } else {
            SRV_TRY(launch_colweights(s->d_col_ptr + r->coff, s->d_cval, s->f32, r->n, r->w_mode,
                                      s->d_w + r->coff, s->d_w + s->Ncap + r->coff,
                                      s->d_wf ? s->d_wf + r->coff : nullptr,
                                      s->d_wf ? s->d_wf + s->Ncap + r->coff : nullptr, st));
        }
    }
    SysState z;
    std::memset(&z, 0, sizeof z);
    z.tol = r->tol;
    z.maxit = r->maxit < 0 ? r->n : r->maxit;
    z.stop_on_true = 1;
    z.inner_tol2 = s->f32 ? 1e-8 : 0.0;
    z.phase = PH_SETUP;
    s->h_st[r->slot] = z;
    SRV_TRY(cudaMemcpyAsync(s->d_st + r->slot, &s->h_st[r->slot], sizeof(SysState), cudaMemcpyHostToDevice, st));
    SRV_TRY(cudaStreamSynchronize(st));   // h_st entry and host vectors may be reused after this
    return true;
}

// Concatenates the resident systems' tiles (slot order) and uploads them
// with the per-slot descriptors.
static bool srv_rebuild(plss_server *s) {
    std::vector<Tile> rt, ct, vt;
    std::vector<int32_t> rfirst, cfirst;   // global first slice of each sliced tile
    for (int32_t i = 0; i < s->Scap; ++i) {
        SrvRequest *r = s->slot_req[size_t(i)];
        SysDesc &d = s->h_desc[size_t(i)];
        std::memset(&d, 0, sizeof d);
        if (!r) continue;
        d.row_off = r->roff;
        d.col_off = r->coff;
        d.m = int32_t(r->m);
        d.n = int32_t(r->n);
        d.rt_begin = int32_t(rt.size());
        for (size_t k = 0; k < r->rt.size(); ++k) {
            const Tile t = r->rt[k];
            rt.push_back({i, t.begin + int32_t(r->roff), t.end + int32_t(r->roff), t.group});
            rfirst.push_back(r->hr.first.empty() ? 0 : int32_t(r->sloff) + r->hr.first[k]);
        }
        d.rt_count = int32_t(rt.size()) - d.rt_begin;
        d.ct_begin = int32_t(ct.size());
        for (size_t k = 0; k < r->ct.size(); ++k) {
            const Tile t = r->ct[k];
            ct.push_back({i, t.begin + int32_t(r->coff), t.end + int32_t(r->coff), t.group});
            cfirst.push_back(r->hc.first.empty() ? 0
                                                 : int32_t(r->sloff + int64_t(r->hr.ptr.size())) + r->hc.first[k]);
        }
        d.ct_count = int32_t(ct.size()) - d.ct_begin;
        d.vt_begin = int32_t(vt.size());
        for (Tile t : r->vt) vt.push_back({i, t.begin + int32_t(r->coff), t.end + int32_t(r->coff), t.group});
        d.vt_count = int32_t(vt.size()) - d.vt_begin;
        r->rt_begin = d.rt_begin;
    }
    cudaStream_t st = s->stream;
    if (!rt.empty()) SRV_TRY(cudaMemcpyAsync(s->d_rt, rt.data(), sizeof(Tile) * rt.size(), cudaMemcpyHostToDevice, st));
    if (!ct.empty()) SRV_TRY(cudaMemcpyAsync(s->d_ct, ct.data(), sizeof(Tile) * ct.size(), cudaMemcpyHostToDevice, st));
    if (!vt.empty()) SRV_TRY(cudaMemcpyAsync(s->d_vt, vt.data(), sizeof(Tile) * vt.size(), cudaMemcpyHostToDevice, st));
    if (s->sliced && !rfirst.empty())
        SRV_TRY(cudaMemcpyAsync(s->d_rfirst, rfirst.data(), 4 * rfirst.size(), cudaMemcpyHostToDevice, st));
    if (s->sliced && !cfirst.empty())
        SRV_TRY(cudaMemcpyAsync(s->d_cfirst, cfirst.data(), 4 * cfirst.size(), cudaMemcpyHostToDevice, st));
    SRV_TRY(cudaMemcpyAsync(s->d_desc, s->h_desc.data(), sizeof(SysDesc) * size_t(s->Scap), cudaMemcpyHostToDevice, st));
    int32_t nact = 0;
    for (int32_t i = 0; i < s->Scap; ++i)
        if (s->slot_req[size_t(i)]) ++nact;
    SRV_TRY(cudaMemcpyAsync(s->d_active, &nact, 4, cudaMemcpyHostToDevice, st));
    SRV_TRY(cudaStreamSynchronize(st));
    return true;
}

static SweepArgs srv_args(plss_server *s) {
    SweepArgs a;
    std::memset(&a, 0, sizeof a);
    a.rsl.g = a.csl.g = 1;   // one lane per segment in the arena's slices
    if (s->sliced) {
        a.rsl.first = s->d_rfirst;
        a.csl.first = s->d_cfirst;
        a.rsl.ptr = a.csl.ptr = s->d_sl_ptr;
        a.rsl.seg = a.csl.seg = s->d_sl_seg;
        a.rsl.idx = a.csl.idx = s->d_sl_idx;
        a.rsl.val = a.csl.val = s->d_sl_val;
    }
    a.row_ptr = s->d_row_ptr;
    a.col_idx = s->d_col_idx;
    a.val = s->d_val;
    a.col_ptr = s->d_col_ptr;
    a.row_idx = s->d_row_idx;
    a.cval = s->d_cval;
    a.rtiles = s->d_rt;
    a.ctiles = s->d_ct;
    a.vtiles = s->d_vt;
    a.n_rtiles = int32_t(s->arena.tiles_r);
    a.n_ctiles = int32_t(s->arena.tiles_c);
    a.n_vtiles = int32_t(s->arena.tiles_v);
    a.desc = s->d_desc;
    a.st = s->d_st;
    a.part_row = s->d_part_row;
    a.part_col = s->d_part_col;
    a.part_upd = s->d_part_upd;
    a.n_active = s->d_active;
    a.b = s->d_b;
    a.x = s->d_x;
    a.r = s->d_r;
    a.p = s->d_p;
    a.u = s->d_u;
    a.w = s->d_w;
    a.winv = s->d_w + s->Ncap;
    a.wf = s->d_wf;
    a.winvf = s->d_wf ? s->d_wf + s->Ncap : nullptr;
    return a;
}

// Result of a finished slot: x, the true residual, status, latency.
static bool srv_retire(plss_server *s, SrvRequest *r) {
    cudaStream_t st = s->stream;
    const SysState &z = s->h_st[r->slot];
    r->x.resize(size_t(r->n));
    if (r->n > 0) SRV_TRY(cudaMemcpyAsync(r->x.data(), s->d_x + r->coff, 8 * size_t(r->n), cudaMemcpyDeviceToHost, st));
    double rel = 0.0;
    if (r->m > 0 && !r->rt.empty()) {
        const int32_t nt = int32_t(r->rt.size());
        SRV_TRY(launch_spmv(s->d_row_ptr, s->d_col_idx, s->d_val, s->f32, s->d_rt + r->rt_begin, nt,
                            s->d_x, s->d_vout, s->d_b, s->d_part_res, std::min(nt, s->nsm * kCtasPerSm), st));
        std::vector<double> part(static_cast<size_t>(nt));
        SRV_TRY(cudaMemcpyAsync(part.data(), s->d_part_res, 8 * size_t(nt), cudaMemcpyDeviceToHost, st));
        SRV_TRY(cudaStreamSynchronize(st));
        double ss = 0.0;
        for (double v : part) ss += v;
        rel = z.nb > 0.0 ? std::sqrt(ss) / z.nb : 0.0;
    } else {
        SRV_TRY(cudaStreamSynchronize(st));
    }
    r->res.status = z.status;
    r->res.reserved = 0;
    r->res.iters = z.iters;
    r->res.relres_rec = z.relres_rec;
    r->res.relres_true = rel;
    r->res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - r->t_submit).count();
    return true;
}

static void srv_fail_all(plss_server *s) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int32_t i = 0; i < s->Scap; ++i) {
        SrvRequest *r = s->slot_req[size_t(i)];
        if (!r) continue;
        r->res.status = PLSS_ERR_CUDA;
        r->x.assign(size_t(r->n), 0.0);
        s->done[r->ticket] = r;
        s->live.erase(r->ticket);
        srv_unplace(s, r);
        s->running -= 1;
    }
}

static void srv_worker(plss_server *s) {
    cudaSetDevice(s->device);
    bool dirty = false;
    while (!s->stop.load()) {
        // admit
        std::vector<SrvRequest *> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (!s->queue.empty()) {
                SrvRequest *r = s->queue.front();
                if (!srv_place(s, r)) break;
                s->queue.pop_front();
                admitted.push_back(r);
                s->running += 1;
            }
            if (admitted.empty() && s->running == 0) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        TraceRange tr("plss server: scheduling round");
        bool ok = true;
        for (SrvRequest *r : admitted) ok = ok && srv_upload(s, r);
        if (ok && (dirty || !admitted.empty())) ok = srv_rebuild(s);
        dirty = false;
        // iterate
        if (ok) {
            const SweepArgs a = srv_args(s);
            const int gr = std::max(1, std::min(a.n_rtiles, s->nsm * sweep_ctas_per_sm(0, s->f32)));
            const int gc = std::max(1, std::min(a.n_ctiles, s->nsm * sweep_ctas_per_sm(1, s->f32)));
            const int gv = std::max(1, std::min(a.n_vtiles, s->nsm * sweep_ctas_per_sm(2, s->f32)));
            for (int i = 0; i < s->so.bodies_per_poll && ok; ++i) {
                ok = launch_col_sweep(a, s->f32, gc, s->stream) == cudaSuccess &&
                     launch_update(a, s->f32, gv, s->stream) == cudaSuccess &&
                     launch_row_sweep(a, s->f32, gr, s->stream) == cudaSuccess;
            }
            if (!ok) s->fatal = "kernel launch failed";
            ok = ok && cudaMemcpyAsync(s->h_st, s->d_st, sizeof(SysState) * size_t(s->Scap),
                                       cudaMemcpyDeviceToHost, s->stream) == cudaSuccess &&
                 cudaStreamSynchronize(s->stream) == cudaSuccess;
            if (!ok && s->fatal.empty()) s->fatal = cudaGetErrorString(cudaGetLastError());
        }
        // retire
        for (int32_t i = 0; ok && i < s->Scap; ++i) {
            SrvRequest *r = s->slot_req[size_t(i)];
            if (!r || s->h_st[i].phase != PH_DONE) continue;
            ok = srv_retire(s, r);
            if (!ok) break;
            std::lock_guard<std::mutex> lk(s->mu);
            srv_unplace(s, r);
            s->done[r->ticket] = r;
            s->live.erase(r->ticket);
            s->running -= 1;
            s->completed += 1;
            dirty = true;
        }
        if (!ok) {
            srv_fail_all(s);
            return;
        }
    }
}

}  // namespace plss

using namespace plss;

extern "C" {

void plss_server_opts_default(plss_server_opts *o) {
    if (!o) return;
    o->max_slots = 64;
    o->max_queue = 4096;
    o->hbm_budget_bytes = 0;
    o->precision = PLSS_FP64;
    o->bodies_per_poll = 8;
    o->layout = PLSS_LAYOUT_CSR;   // measured faster for serving (see plss.h)
    o->reserved = 0;
}

plss_status plss_server_create(const plss_server_opts *so_in, plss_server **out) {
    clear_error();
    if (!out) return fail(PLSS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    plss_server_opts so;
    plss_server_opts_default(&so);
    if (so_in) so = *so_in;
    if (so.max_slots < 1 || so.max_queue < 1 || so.bodies_per_poll < 1)
        return fail(PLSS_ERR_INVALID, "max_slots, max_queue and bodies_per_poll must be positive");
    if (so.precision != PLSS_FP64 && so.precision != PLSS_FP32) return fail(PLSS_ERR_INVALID, "unknown precision");
    if (so.layout != PLSS_LAYOUT_AUTO && so.layout != PLSS_LAYOUT_CSR) return fail(PLSS_ERR_INVALID, "unknown layout");
    plss_server *s = new plss_server();
    s->so = so;
    s->f32 = so.precision == PLSS_FP32;
    s->sliced = so.layout == PLSS_LAYOUT_AUTO;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(PLSS_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    int64_t budget = so.hbm_budget_bytes > 0 ? so.hbm_budget_bytes : (int64_t(4) << 30);
    budget = std::min<int64_t>(budget, int64_t(double(free_b) * 0.8));
    // arena: nonzeros twice (CSR and transpose), rows (row_ptr, b, r, partials)
    // and columns (col_ptr, x, p, u, w) sized for up to 2 columns and 1 row
    // per 8 nonzeros
    const int64_t sb = s->f32 ? 4 : 8;
    s->bytes_per_nnz = 2 * (4 + sb);
    s->bytes_per_row = 4 + 8 + sb + 8 + 24;
    s->bytes_per_col = 4 + 8 + 2 * sb + 8 + 8;
    // sliced copies (AUTO): at most 5/4 of the nonzeros per side, and one
    // slice slot (offset + 32 slot ids) per 32 rows or columns
    if (s->sliced) {
        s->bytes_per_nnz += 2 * (4 + sb) * 5 / 4;
        s->bytes_per_row += 4;
        s->bytes_per_col += 4;
    }
    const double per_nnz = double(s->bytes_per_nnz) + double(s->bytes_per_row) / 8.0 + 2.0 * double(s->bytes_per_col) / 8.0;
    s->Zcap = std::min<int64_t>(int64_t(double(budget) / per_nnz), INT32_MAX / 2);
    s->Mcap = std::min<int64_t>(s->Zcap / 8 + 64 * so.max_slots, INT32_MAX / 2);
    s->Ncap = std::min<int64_t>(2 * (s->Zcap / 8) + 64 * so.max_slots, INT32_MAX / 2);
    s->Scap = so.max_slots;
    s->Tr = 2 * (s->Zcap / 1024) + s->Mcap / kTileMaxSegs + 2 * int64_t(s->Scap) + 16;
    s->Tc = 2 * (s->Zcap / 1024) + s->Ncap / kTileMaxSegs + 2 * int64_t(s->Scap) + 16;
    s->Tv = s->Ncap / kVecTile + 2 * int64_t(s->Scap) + 16;
    if (s->sliced) {
        // a request's slices take (m + 31)/32 + (n + 31)/32 + 2 slots and its
        // elements at most 5/4 of 2 nnz plus one slice row of 32 per tile
        s->SLcap = (s->Mcap + s->Ncap) / 32 + 4 * int64_t(so.max_slots) + 64;
        s->ELcap = s->Zcap * 5 / 2 + 32 * (s->Tr + s->Tc) + 1024;
    }
    s->arena.init(s->Scap, s->Mcap, s->Ncap, s->Zcap, s->SLcap, s->ELcap, s->Tr, s->Tc, s->Tv);
    s->h_desc.assign(size_t(s->Scap), SysDesc{});
    s->slot_req.assign(size_t(s->Scap), nullptr);
    plss_status st = PLSS_OK;
    auto A = [&](void **p, size_t bytes, const char *w) {
        if (st == PLSS_OK) st = dalloc(p, bytes, w);
    };
    A(reinterpret_cast<void **>(&s->d_row_ptr), 4 * size_t(s->Mcap), "arena row_ptr");
    A(reinterpret_cast<void **>(&s->d_col_idx), 4 * size_t(s->Zcap), "arena col_idx");
    A(&s->d_val, size_t(sb) * size_t(s->Zcap), "arena val");
    A(reinterpret_cast<void **>(&s->d_col_ptr), 4 * size_t(s->Ncap), "arena col_ptr");
    A(reinterpret_cast<void **>(&s->d_row_idx), 4 * size_t(s->Zcap), "arena row_idx");
    A(&s->d_cval, size_t(sb) * size_t(s->Zcap), "arena cval");
    A(reinterpret_cast<void **>(&s->d_b), 8 * size_t(s->Mcap), "arena b");
    A(&s->d_r, size_t(sb) * size_t(s->Mcap), "arena r");
    A(reinterpret_cast<void **>(&s->d_vout), 8 * size_t(s->Mcap), "arena tmp");
    A(reinterpret_cast<void **>(&s->d_x), 8 * size_t(s->Ncap), "arena x");
    A(&s->d_p, size_t(sb) * size_t(s->Ncap), "arena p");
    A(&s->d_u, size_t(sb) * size_t(s->Ncap), "arena u");
    A(reinterpret_cast<void **>(&s->d_w), 16 * size_t(s->Ncap), "arena w");   // w, then 1/w
    if (s->f32) A(reinterpret_cast<void **>(&s->d_wf), 8 * size_t(s->Ncap), "arena wf");
    A(reinterpret_cast<void **>(&s->d_part_row), 16 * size_t(s->Tr), "partials");
    A(reinterpret_cast<void **>(&s->d_part_res), 8 * size_t(s->Tr), "partials");
    A(reinterpret_cast<void **>(&s->d_part_col), 8 * size_t(s->Tc), "partials");
    A(reinterpret_cast<void **>(&s->d_part_upd), 8 * size_t(s->Tv), "partials");
    A(reinterpret_cast<void **>(&s->d_rt), sizeof(Tile) * size_t(s->Tr), "tiles");
    A(reinterpret_cast<void **>(&s->d_ct), sizeof(Tile) * size_t(s->Tc), "tiles");
    A(reinterpret_cast<void **>(&s->d_vt), sizeof(Tile) * size_t(s->Tv), "tiles");
    A(reinterpret_cast<void **>(&s->d_desc), sizeof(SysDesc) * size_t(s->Scap), "desc");
    A(reinterpret_cast<void **>(&s->d_st), sizeof(SysState) * size_t(s->Scap), "state");
    A(reinterpret_cast<void **>(&s->d_active), 16, "active");
    if (s->sliced) {
        A(reinterpret_cast<void **>(&s->d_sl_ptr), 4 * size_t(s->SLcap), "arena slice offsets");
        A(reinterpret_cast<void **>(&s->d_sl_seg), 128 * size_t(s->SLcap), "arena slice slots");
        A(reinterpret_cast<void **>(&s->d_sl_idx), 4 * size_t(s->ELcap), "arena sliced indices");
        A(&s->d_sl_val, size_t(sb) * size_t(s->ELcap), "arena sliced values");
        A(reinterpret_cast<void **>(&s->d_rfirst), 4 * size_t(s->Tr), "arena sliced tiles");
        A(reinterpret_cast<void **>(&s->d_cfirst), 4 * size_t(s->Tc), "arena sliced tiles");
    }
    if (st == PLSS_OK && (cudaMallocHost(reinterpret_cast<void **>(&s->h_st), sizeof(SysState) * size_t(s->Scap)) != cudaSuccess ||
                          cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaMemset(s->d_st, 0, sizeof(SysState) * size_t(s->Scap)) != cudaSuccess ||
                          cudaMemset(s->d_p, 0, size_t(sb) * size_t(s->Ncap)) != cudaSuccess))
        st = fail(PLSS_ERR_CUDA, "server set-up failed");
    if (st != PLSS_OK) {
        srv_free_device(s);
        delete s;
        return st;
    }
    std::memset(s->h_st, 0, sizeof(SysState) * size_t(s->Scap));
    s->worker = std::thread(srv_worker, s);
    *out = s;
    return PLSS_OK;
}

plss_status plss_submit(plss_server *s, const plss_csr *A, const double *b, const double *x0,
                        const plss_opts *o, uint64_t *ticket) {
    clear_error();
    if (!s || !ticket) return fail(PLSS_ERR_INVALID, "NULL server or ticket");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    plss_status st = check_opts(o);
    if (st != PLSS_OK) return st;
    if (o->sketch != PLSS_SKETCH_RESIDUAL) return fail(PLSS_ERR_INVALID, "the server runs the residual sketch");
    if (o->w_mode < 0 || o->w_mode > 2) return fail(PLSS_ERR_INVALID, "unknown w_mode");
    HostCsr h;
    if ((st = fetch_csr(A, h)) != PLSS_OK) return st;
    if (h.m > 0 && !b) return fail(PLSS_ERR_INVALID, "b is NULL");
    SrvRequest *r = new SrvRequest();
    srv_prepare(s, h, r);
    r->b.assign(b, b + r->m);
    if (x0) r->x0.assign(x0, x0 + r->n);
    r->tol = o->tol;
    r->maxit = o->maxit;
    r->w_mode = o->w_mode;
    if (!s->arena.ever_fits(r->need())) {
        delete r;
        return fail(PLSS_ERR_BUSY, "request larger than the server arena");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->fatal.empty()) {
        delete r;
        return fail(PLSS_ERR_CUDA, "server stopped: %s", s->fatal.c_str());
    }
    if (int64_t(s->queue.size()) >= s->so.max_queue) {
        delete r;
        return fail(PLSS_ERR_BUSY, "queue full (%d requests)", s->so.max_queue);
    }
    r->ticket = s->next_ticket++;
    r->t_submit = std::chrono::steady_clock::now();
    s->queue.push_back(r);
    s->live[r->ticket] = 1;
    *ticket = r->ticket;
    s->cv.notify_one();
    return PLSS_OK;
}

plss_status plss_poll(plss_server *s, uint64_t ticket, double *x_out, plss_result *res) {
    clear_error();
    if (!s) return fail(PLSS_ERR_INVALID, "NULL server");
    SrvRequest *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->done.find(ticket);
        if (it == s->done.end()) {
            if (s->live.count(ticket)) return PLSS_PENDING;
            return fail(PLSS_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
        }
        r = it->second;
        s->done.erase(it);
    }
    if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), 8 * r->x.size());
    if (res) *res = r->res;
    const plss_status out = plss_status(r->res.status);
    delete r;
    return out;
}

plss_status plss_server_stats(plss_server *s, int64_t *completed, int64_t *queued, int64_t *running,
                              int64_t *bytes_in_use) {
    clear_error();
    if (!s) return fail(PLSS_ERR_INVALID, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (queued) *queued = int64_t(s->queue.size());
    if (running) *running = s->running;
    if (bytes_in_use)
        *bytes_in_use = s->arena.nnzs.used * s->bytes_per_nnz + s->arena.rows.used * s->bytes_per_row +
                        s->arena.cols.used * s->bytes_per_col;
    return PLSS_OK;
}

void plss_server_destroy(plss_server *s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->stream);
    for (SrvRequest *r : s->queue) delete r;
    for (auto &kv : s->done) delete kv.second;
    for (SrvRequest *r : s->slot_req) delete r;
    srv_free_device(s);
    delete s;
}

}  // extern "C"
