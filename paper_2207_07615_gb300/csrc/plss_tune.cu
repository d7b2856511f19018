// plss_tune.cu -- plss_tune: the sweep plan of a matrix (or a batch of
// them) chosen by measurement. Host code over the library's own entry
// points; the plan itself is built in plss_plan.cu and the candidates differ
// only in the knobs that plan exposes (layout, tile size, schedule).
#include <chrono>
#include <cstring>
#include <vector>

#include "plss_ctx.h"
#include "plss_launch.h"
#include "plss_trace.h"

using namespace plss;

namespace {

struct DevVec {
    double *p = nullptr;
    ~DevVec() { dfree(p); }
};

struct CtxHold {
    plss_ctx *c = nullptr;
    ~CtxHold() {
        if (c) plss_destroy(c);
    }
};

// Builds the candidate context `co`, then for each schedule it allows runs
// one untimed and one timed solve of exactly `updates` updates on b = A 1
// and appends what it measured.
plss_status measure(const plss_csr *As, int32_t nsys, const plss_opts &co, int32_t updates,
                    std::vector<plss_tune_entry> &table) {
    CtxHold h;
    plss_status st = plss_create_batched(As, nsys, &co, &h.c);
    if (st == PLSS_ERR_NOMEM) {
        table.push_back({co.layout, co.tile_shift, PLSS_SCHED_GRID, int32_t(st), 0.0});
        return PLSS_OK;
    }
    if (st != PLSS_OK) return st;
    plss_ctx *c = h.c;
    cudaStream_t s = static_cast<cudaStream_t>(co.stream);

    DevVec ones, b, x;
    const size_t nb = size_t(std::max<int64_t>(c->m, 1)), nx = size_t(std::max<int64_t>(c->n, 1));
    st = dalloc(reinterpret_cast<void **>(&ones.p), 8 * nx, "tune ones");
    if (st == PLSS_OK) st = dalloc(reinterpret_cast<void **>(&b.p), 8 * nb, "tune b");
    if (st == PLSS_OK) st = dalloc(reinterpret_cast<void **>(&x.p), 8 * nx, "tune x");
    if (st == PLSS_ERR_NOMEM) {
        table.push_back({co.layout, co.tile_shift, PLSS_SCHED_GRID, int32_t(st), 0.0});
        return PLSS_OK;
    }
    if (st != PLSS_OK) return st;
    const std::vector<double> h_ones(nx, 1.0);
    if (cudaMemcpyAsync(ones.p, h_ones.data(), 8 * nx, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "tune: copy of the ones vector failed");
    // b = A 1 over the packed (block-diagonal) systems: consistent for each
    if (launch_spmv(c->d_row_ptr, c->d_col_idx, c->d_val, c->f32, c->d_rt, int32_t(c->h_rt.size()), ones.p, b.p,
                    nullptr, nullptr, c->grid_r, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "tune: b = A 1 failed: %s", cudaGetErrorString(cudaGetLastError()));

    std::vector<const double *> bp(static_cast<size_t>(nsys));
    std::vector<double *> xp(static_cast<size_t>(nsys));
    for (int32_t i = 0; i < nsys; ++i) {
        bp[size_t(i)] = b.p + c->h_desc[size_t(i)].row_off;
        xp[size_t(i)] = x.p + c->h_desc[size_t(i)].col_off;
    }
    std::vector<plss_result> res(static_cast<size_t>(nsys));
    std::vector<int32_t> schedules = {PLSS_SCHED_GRID};
    if (c->small_fits) schedules.push_back(PLSS_SCHED_SMALL);
    for (int32_t sched : schedules) {
        plss_opts so = co;
        so.sketch = PLSS_SKETCH_RESIDUAL;
        so.schedule = sched;
        so.tol = 0.0;
        so.maxit = updates;
        so.io_device = 1;
        so.hist = nullptr;
        so.hist_cap = 0;
        so.profile = 0;
        double us = 0.0;
        for (int rep = 0; rep < 2; ++rep) {   // untimed (graphs, weights), then timed
            const auto t0 = std::chrono::steady_clock::now();
            st = plss_solve_batched(c, bp.data(), nullptr, xp.data(), &so, res.data());
            const auto t1 = std::chrono::steady_clock::now();
            if (st != PLSS_OK && st != PLSS_NOT_CONVERGED && st != PLSS_ERR_BREAKDOWN) return st;
            int64_t it = 0;
            for (const plss_result &r : res) it = std::max<int64_t>(it, r.iters);
            us = std::chrono::duration<double, std::micro>(t1 - t0).count() / double(std::max<int64_t>(it, 1));
        }
        table.push_back({co.layout, co.tile_shift, sched, int32_t(PLSS_OK), us});
    }
    return PLSS_OK;
}

}  // namespace

extern "C" plss_status plss_tune(const plss_csr *As, int32_t nsys, const plss_opts *o, int32_t updates,
                                 plss_opts *best, plss_tune_entry *entries, int32_t cap, int32_t *count) {
    clear_error();
    if (!As || !best || !count) return fail(PLSS_ERR_INVALID, "As, best and count must not be NULL");
    if (nsys <= 0) return fail(PLSS_ERR_INVALID, "nsys must be positive");
    if (updates < 1 || updates > 100000) return fail(PLSS_ERR_INVALID, "updates %d outside [1, 100000]", updates);
    if (cap < 0 || (cap > 0 && !entries)) return fail(PLSS_ERR_INVALID, "entries NULL with cap %d", cap);
    plss_opts base;
    plss_opts_default(&base);
    if (o) base = *o;

    TraceRange tr("plss: tune");
    std::vector<plss_tune_entry> table;
    for (int32_t layout : {PLSS_LAYOUT_AUTO, PLSS_LAYOUT_CSR}) {
        for (int32_t shift : {-1, 0, 1}) {
            plss_opts co = base;
            co.layout = layout;
            co.tile_shift = shift;
            const plss_status st = measure(As, nsys, co, updates, table);
            if (st != PLSS_OK) return st;
        }
    }
    const plss_tune_entry *win = nullptr;
    for (const plss_tune_entry &e : table)
        if (e.status == PLSS_OK && (!win || e.us_per_update < win->us_per_update)) win = &e;
    *count = int32_t(table.size());
    if (cap > 0)
        std::memcpy(entries, table.data(), sizeof(plss_tune_entry) * size_t(std::min<int64_t>(cap, table.size())));
    if (!win) return fail(PLSS_ERR_NOMEM, "tune: no candidate plan fits in device memory");
    *best = base;
    best->layout = win->layout;
    best->tile_shift = win->tile_shift;
    best->schedule = win->schedule;
    clear_error();
    return PLSS_OK;
}
