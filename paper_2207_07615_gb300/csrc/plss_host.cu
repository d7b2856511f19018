// plss_host.cu -- C ABI of libplss: validation, packing, tile schedules,
// device memory, the CUDA-graph iteration driver and results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "plss.h"
#include "plss_ctx.h"
#include "plss_dev.cuh"
#include "plss_launch.h"
#include "plss_trace.h"

namespace plss {

static thread_local std::string g_err;

plss_status fail(plss_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

void clear_error() { g_err.clear(); }
const char *last_error() { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// Tile schedules (tiles, sliced copies and warp ranges: plss_plan.cu)
// ---------------------------------------------------------------------------

PlanSlots plan_slots(int nsm) {
    PlanSlots p;
    p.f64 = int64_t(nsm) * std::max(sweep_ctas_per_sm(0, false), sweep_ctas_per_sm(1, false));
    p.f32 = int64_t(nsm) * std::max(sweep_ctas_per_sm(0, true), sweep_ctas_per_sm(1, true));
    return p;
}

// ---------------------------------------------------------------------------
// Validation and packing
// ---------------------------------------------------------------------------

plss_status fetch_csr(const plss_csr *A, HostCsr &h) {
    if (!A) return fail(PLSS_ERR_INVALID, "A is NULL");
    if (A->m < 0 || A->n < 0 || A->nnz < 0)
        return fail(PLSS_ERR_INVALID, "negative size (m=%lld n=%lld nnz=%lld)", (long long)A->m,
                    (long long)A->n, (long long)A->nnz);
    if (A->m >= INT32_MAX || A->n >= INT32_MAX || A->nnz >= INT32_MAX)
        return fail(PLSS_ERR_INVALID, "sizes above 2^31-1 are not supported");
    if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val)))
        return fail(PLSS_ERR_INVALID, "NULL CSR array");
    h.m = A->m;
    h.n = A->n;
    h.nnz = A->nnz;
    h.row_ptr.resize(size_t(A->m + 1));
    h.col_idx.resize(size_t(A->nnz));
    h.val.resize(size_t(A->nnz));
    // host input: plain copies (no CUDA call, so validation works anywhere)
    auto fetch = [&](void *dst, const void *src, size_t bytes) -> bool {
        if (bytes == 0) return true;
        if (!A->on_device) {
            std::memcpy(dst, src, bytes);
            return true;
        }
        return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    if (!fetch(h.row_ptr.data(), A->row_ptr, size_t(A->m + 1) * 8))
        return fail(PLSS_ERR_CUDA, "copying row_ptr failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (!fetch(h.col_idx.data(), A->col_idx, size_t(A->nnz) * 4))
        return fail(PLSS_ERR_CUDA, "copying col_idx failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (A->val_f32) {
        std::vector<float> tmp(static_cast<size_t>(A->nnz));
        if (!fetch(tmp.data(), A->val, size_t(A->nnz) * 4))
            return fail(PLSS_ERR_CUDA, "copying val failed: %s", cudaGetErrorString(cudaGetLastError()));
        for (size_t k = 0; k < tmp.size(); ++k) h.val[k] = double(tmp[k]);
    } else if (!fetch(h.val.data(), A->val, size_t(A->nnz) * 8)) {
        return fail(PLSS_ERR_CUDA, "copying val failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    // structure checks
    if (h.row_ptr[0] != 0) return fail(PLSS_ERR_INVALID, "row_ptr[0] = %lld, expected 0", (long long)h.row_ptr[0]);
    if (h.row_ptr[size_t(h.m)] != h.nnz)
        return fail(PLSS_ERR_INVALID, "row_ptr[m] = %lld, expected nnz = %lld",
                    (long long)h.row_ptr[size_t(h.m)], (long long)h.nnz);
    for (int64_t i = 0; i < h.m; ++i)
        if (h.row_ptr[size_t(i + 1)] < h.row_ptr[size_t(i)])
            return fail(PLSS_ERR_INVALID, "row_ptr decreases at row %lld", (long long)i);
    for (int64_t i = 0; i < h.m; ++i) {
        const int64_t s = h.row_ptr[size_t(i)], e = h.row_ptr[size_t(i + 1)];
        for (int64_t k = s; k < e; ++k) {
            const int32_t c = h.col_idx[size_t(k)];
            if (c < 0 || c >= h.n)
                return fail(PLSS_ERR_INVALID, "col_idx[%lld] = %d outside [0, %lld)", (long long)k, c,
                            (long long)h.n);
            if (k > s && c <= h.col_idx[size_t(k - 1)])
                return fail(PLSS_ERR_INVALID, "columns not strictly increasing in row %lld", (long long)i);
        }
    }
    for (int64_t k = 0; k < h.nnz; ++k)
        if (!std::isfinite(h.val[size_t(k)]))
            return fail(PLSS_ERR_INVALID, "non-finite value at nonzero %lld", (long long)k);
    return PLSS_OK;
}

// ---------------------------------------------------------------------------
// Device memory helpers
// ---------------------------------------------------------------------------

plss_status dalloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? PLSS_ERR_NOMEM : PLSS_ERR_CUDA,
                    "cudaMalloc(%s, %zu bytes): %s", what, bytes, cudaGetErrorString(e));
    }
    return PLSS_OK;
}

template <typename T>
plss_status upload(T **dst, const std::vector<T> &src, const char *what) {
    plss_status s = dalloc(reinterpret_cast<void **>(dst), src.size() * sizeof(T), what);
    if (s != PLSS_OK) return s;
    if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(PLSS_ERR_CUDA, "upload of %s failed", what);
    return PLSS_OK;
}

// Device copy of a sliced side (all pointers null when no tile is sliced).
static plss_status upload_sliced(const HostSliced &h, Sliced &d, bool f32) {
    d = Sliced{};
    d.g = h.g;
    if (h.seg.empty()) return PLSS_OK;
    int32_t *first = nullptr, *ptr = nullptr, *seg = nullptr, *idx = nullptr;
    plss_status st = upload(&first, h.first, "sliced tiles");
    d.first = first;
    if (st == PLSS_OK) st = upload(&ptr, h.ptr, "slice offsets");
    d.ptr = ptr;
    if (st == PLSS_OK) st = upload(&seg, h.seg, "slice slots");
    d.seg = seg;
    if (st == PLSS_OK) st = upload(&idx, h.idx, "sliced indices");
    d.idx = idx;
    if (st == PLSS_OK) {
        if (f32) {
            float *v = nullptr;
            st = upload(&v, h.v32, "sliced values");
            d.val = v;
        } else {
            double *v = nullptr;
            st = upload(&v, h.v64, "sliced values");
            d.val = v;
        }
    }
    return st;
}

// Uploads the warp ranges of a side (see warp_ranges); *out stays null
// unless every tile is sliced.
static plss_status upload_warp_ranges(const std::vector<Tile> &tiles, const std::vector<int32_t> &sptr,
                                      int64_t nwarps, int32_t **out) {
    *out = nullptr;
    const std::vector<int32_t> wr = warp_ranges(tiles, sptr, nwarps);
    if (wr.empty()) return PLSS_OK;
    return upload(out, wr, "warp ranges");
}

static void free_sliced(Sliced &d) {
    const void *ptrs[] = {d.first, d.ptr, d.seg, d.idx, d.val};
    for (const void *p : ptrs) dfree(const_cast<void *>(p));
    d = Sliced{};
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

#define CUDA_TRY(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return fail(PLSS_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                               \
        }                                                                                        \
    } while (0)

// ---------------------------------------------------------------------------
// Context creation
// ---------------------------------------------------------------------------

static void ctx_free(plss_ctx *c) {
    if (!c) return;
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    for (cudaEvent_t ev : c->prof_ev) cudaEventDestroy(ev);
    c->prof_ev.clear();
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    void *ptrs[] = {c->d_row_ptr, c->d_col_idx, c->d_val, c->d_rt, c->d_ct, c->d_vt, c->d_desc,
                    c->d_st, c->d_part_row, c->d_part_col, c->d_part_upd, c->d_part_res, c->d_active,
                    c->d_b, c->d_x, c->d_w, c->d_wf, c->d_r, c->d_p, c->d_u, c->d_hist, c->d_vin, c->d_vout};
    for (void *p : ptrs) dfree(p);
    if (!c->symmetric) {
        dfree(c->d_col_ptr);
        dfree(c->d_row_idx);
        dfree(c->d_cval);
    }
    free_sliced(c->rsl);
    if (!c->symmetric) free_sliced(c->csl);
    dfree(c->d_rwr);
    dfree(c->d_cwr);
    dfree(c->d_coop_rwr);
    dfree(c->d_coop_cwr);
    dfree(c->d_coop_part);
    dfree(c->d_coop_bar);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->h_active) cudaFreeHost(c->h_active);
    free_extra(c);
    delete c;
}

static plss_status ctx_build(const plss_csr *As, int32_t nsys, const plss_opts *o, plss_ctx **out) {
    TraceRange tr("plss: create context");
    *out = nullptr;
    if (nsys <= 0) return fail(PLSS_ERR_INVALID, "nsys must be positive");
    if (!As) return fail(PLSS_ERR_INVALID, "A is NULL");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    if (o->precision != PLSS_FP64 && o->precision != PLSS_FP32)
        return fail(PLSS_ERR_INVALID, "unknown precision %d", o->precision);
    if (o->layout != PLSS_LAYOUT_AUTO && o->layout != PLSS_LAYOUT_CSR)
        return fail(PLSS_ERR_INVALID, "unknown layout %d", o->layout);
    if (o->tile_shift < -2 || o->tile_shift > 2)
        return fail(PLSS_ERR_INVALID, "tile_shift %d outside [-2, 2]", o->tile_shift);

    std::vector<HostCsr> hs(static_cast<size_t>(nsys));
    int64_t M = 0, N = 0, NNZ = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        plss_status st = fetch_csr(&As[s], hs[size_t(s)]);
        if (st != PLSS_OK) {
            if (nsys > 1) return fail(st, "system %d: %s", s, last_error());
            return st;
        }
        M += hs[size_t(s)].m;
        N += hs[size_t(s)].n;
        NNZ += hs[size_t(s)].nnz;
    }
    if (M >= INT32_MAX || N >= INT32_MAX || NNZ >= INT32_MAX)
        return fail(PLSS_ERR_INVALID, "packed sizes above 2^31-1 are not supported");
    const bool sym = o->symmetric != 0;
    if (sym) {
        for (int32_t s = 0; s < nsys; ++s)
            if (hs[size_t(s)].m != hs[size_t(s)].n)
                return fail(PLSS_ERR_INVALID, "symmetric requires square systems");
    }

    plss_ctx *c = new plss_ctx();
    c->nsys = nsys;
    c->m = M;
    c->n = N;
    c->nnz = NNZ;
    c->f32 = o->precision == PLSS_FP32;
    c->symmetric = sym;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(PLSS_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (c->nsm <= 0) c->nsm = 1;

    // pack (block diagonal, global column indices)
    std::vector<int32_t> rp(static_cast<size_t>(M + 1));
    std::vector<int32_t> ci(static_cast<size_t>(NNZ));
    std::vector<double> v64;
    std::vector<float> v32;
    if (c->f32) v32.resize(size_t(NNZ)); else v64.resize(size_t(NNZ));
    c->h_desc.resize(size_t(nsys));
    int64_t ro = 0, co = 0, zo = 0;
    rp[0] = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        const HostCsr &h = hs[size_t(s)];
        SysDesc &d = c->h_desc[size_t(s)];
        d.row_off = ro;
        d.col_off = co;
        d.m = int32_t(h.m);
        d.n = int32_t(h.n);
        for (int64_t i = 0; i < h.m; ++i) rp[size_t(ro + i + 1)] = int32_t(zo + h.row_ptr[size_t(i + 1)]);
        for (int64_t k = 0; k < h.nnz; ++k) {
            ci[size_t(zo + k)] = int32_t(co + h.col_idx[size_t(k)]);
            if (c->f32) v32[size_t(zo + k)] = float(h.val[size_t(k)]);
            else v64[size_t(zo + k)] = h.val[size_t(k)];
        }
        ro += h.m;
        co += h.n;
        zo += h.nnz;
    }
    hs.clear();

    // transpose (stable counting sort: rows ascending inside each column)
    std::vector<int32_t> cp, ri;
    std::vector<double> cv64;
    std::vector<float> cv32;
    if (!sym) {
        cp.assign(size_t(N + 1), 0);
        ri.resize(size_t(NNZ));
        if (c->f32) cv32.resize(size_t(NNZ)); else cv64.resize(size_t(NNZ));
        for (int64_t k = 0; k < NNZ; ++k) cp[size_t(ci[size_t(k)] + 1)] += 1;
        for (int64_t j = 0; j < N; ++j) cp[size_t(j + 1)] += cp[size_t(j)];
        std::vector<int32_t> next(cp.begin(), cp.end() - 1);
        for (int64_t i = 0; i < M; ++i)
            for (int32_t k = rp[size_t(i)]; k < rp[size_t(i + 1)]; ++k) {
                const int32_t dst = next[size_t(ci[size_t(k)])]++;
                ri[size_t(dst)] = int32_t(i);
                if (c->f32) cv32[size_t(dst)] = v32[size_t(k)]; else cv64[size_t(dst)] = v64[size_t(k)];
            }
    }
    const int32_t *colp = sym ? rp.data() : cp.data();

    // sliced copies unless the caller asks for the plain layout (or the
    // padded copy could overflow 32-bit offsets)
    const bool slice = o->layout == PLSS_LAYOUT_AUTO && NNZ < 1800000000;
    const int32_t g_r = slice_lanes(NNZ, M), g_c = sym ? g_r : slice_lanes(NNZ, N);
    PlanSlots slots = plan_slots(c->nsm);
    slots.shift = o->tile_shift;
    for (int32_t s = 0; s < nsys; ++s) {
        SysDesc &d = c->h_desc[size_t(s)];
        d.rt_begin = int32_t(c->h_rt.size());
        build_side(rp.data(), d.row_off, d.row_off + d.m, s, NNZ, slots, c->f32, slice, g_r, c->h_rt);
        d.rt_count = int32_t(c->h_rt.size()) - d.rt_begin;
        d.ct_begin = int32_t(c->h_ct.size());
        build_side(colp, d.col_off, d.col_off + d.n, s, NNZ, slots, c->f32, slice, g_c, c->h_ct);
        d.ct_count = int32_t(c->h_ct.size()) - d.ct_begin;
        d.vt_begin = int32_t(c->h_vt.size());
        build_vec_tiles(d.col_off, d.col_off + d.n, s, kVecTile, c->h_vt);
        d.vt_count = int32_t(c->h_vt.size()) - d.vt_begin;
    }

    plss_status st = PLSS_OK;
#define TRY_ST(x)                  \
    do {                           \
        st = (x);                  \
        if (st != PLSS_OK) {       \
            ctx_free(c);           \
            return st;             \
        }                          \
    } while (0)
    TRY_ST(upload(&c->d_row_ptr, rp, "row_ptr"));
    TRY_ST(upload(&c->d_col_idx, ci, "col_idx"));
    if (c->f32) TRY_ST(upload(reinterpret_cast<float **>(&c->d_val), v32, "val"));
    else TRY_ST(upload(reinterpret_cast<double **>(&c->d_val), v64, "val"));
    if (sym) {
        c->d_col_ptr = c->d_row_ptr;
        c->d_row_idx = c->d_col_idx;
        c->d_cval = c->d_val;
    } else {
        TRY_ST(upload(&c->d_col_ptr, cp, "col_ptr"));
        TRY_ST(upload(&c->d_row_idx, ri, "row_idx"));
        if (c->f32) TRY_ST(upload(reinterpret_cast<float **>(&c->d_cval), cv32, "cval"));
        else TRY_ST(upload(reinterpret_cast<double **>(&c->d_cval), cv64, "cval"));
    }
    // A single system whose side is sliced throughout runs that side's sweep
    // over warp ranges of slices, where tiles play no part: its slices are
    // then cut from all segments sorted by length (less padding than
    // tile-local sorting).
    auto all_sliced = [](const std::vector<Tile> &ts) {
        if (ts.empty()) return false;
        for (const Tile &t : ts)
            if (!(t.group & kSliced)) return false;
        return true;
    };
    auto fill_side = [&](const int32_t *ptr, const int32_t *idx, const double *vd, const float *vf,
                         const std::vector<Tile> &ts, int64_t nseg, int32_t g, HostSliced &out) {
        if (nsys == 1 && all_sliced(ts) && nseg > 0) {
            const std::vector<Tile> whole = {Tile{0, 0, int32_t(nseg), ts[0].group}};
            fill_sliced(ptr, idx, vd, vf, whole, g, out);
            out.first.assign(ts.size(), 0);
        } else {
            fill_sliced(ptr, idx, vd, vf, ts, g, out);
        }
    };
    HostSliced hsl;
    fill_side(rp.data(), ci.data(), c->f32 ? nullptr : v64.data(), c->f32 ? v32.data() : nullptr, c->h_rt, M, g_r,
              hsl);
    TRY_ST(upload_sliced(hsl, c->rsl, c->f32));
    c->sl_elems[0] = int64_t(hsl.idx.size());
    const std::vector<int32_t> rsl_ptr = hsl.ptr;
    std::vector<int32_t> csl_ptr;
    if (sym) {
        c->csl = c->rsl;   // same tiles over the same arrays
        c->sl_elems[1] = c->sl_elems[0];
        csl_ptr = rsl_ptr;
    } else {
        fill_side(cp.data(), ri.data(), c->f32 ? nullptr : cv64.data(), c->f32 ? cv32.data() : nullptr, c->h_ct, N,
                  g_c, hsl);
        TRY_ST(upload_sliced(hsl, c->csl, c->f32));
        c->sl_elems[1] = int64_t(hsl.idx.size());
        csl_ptr = hsl.ptr;
    }
    hsl = HostSliced();
    TRY_ST(upload(&c->d_rt, c->h_rt, "row tiles"));
    TRY_ST(upload(&c->d_ct, c->h_ct, "col tiles"));
    TRY_ST(upload(&c->d_vt, c->h_vt, "vec tiles"));
    TRY_ST(upload(&c->d_desc, c->h_desc, "desc"));
    const size_t sb = c->f32 ? 4 : 8;
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_st), sizeof(SysState) * size_t(nsys), "state"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_part_row), 16 * c->h_rt.size(), "partials"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_part_col), 8 * c->h_ct.size(), "partials"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_part_upd), 8 * c->h_vt.size(), "partials"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_part_res), 8 * c->h_rt.size(), "partials"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_active), 16, "counter"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_b), 8 * size_t(M), "b"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_x), 8 * size_t(N), "x"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_w), 16 * size_t(N), "w"));   // w, then 1/w
    if (c->f32) TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_wf), 8 * size_t(N), "wf"));   // float copies
    TRY_ST(dalloc(&c->d_r, sb * size_t(M), "r"));
    TRY_ST(dalloc(&c->d_p, sb * size_t(N), "p"));
    TRY_ST(dalloc(&c->d_u, sb * size_t(N), "u"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_vin), 8 * size_t(std::max(M, N)), "tmp"));
    TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_vout), 8 * size_t(std::max(M, N)), "tmp"));
    if (cudaMemset(c->d_st, 0, sizeof(SysState) * size_t(nsys)) != cudaSuccess ||
        cudaMemset(c->d_p, 0, sb * size_t(N)) != cudaSuccess) {
        ctx_free(c);
        return fail(PLSS_ERR_CUDA, "cudaMemset failed");
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&c->h_st), sizeof(SysState) * size_t(nsys)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&c->h_active), 16) != cudaSuccess) {
        ctx_free(c);
        return fail(PLSS_ERR_NOMEM, "pinned host allocation failed");
    }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        ctx_free(c);
        return fail(PLSS_ERR_CUDA, "stream/event creation failed");
    }
    c->grid_r = std::max(1, std::min(int(c->h_rt.size()), c->nsm * sweep_ctas_per_sm(0, c->f32)));
    c->grid_c = std::max(1, std::min(int(c->h_ct.size()), c->nsm * sweep_ctas_per_sm(1, c->f32)));
    c->grid_v = std::max(1, std::min(int(c->h_vt.size()), c->nsm * sweep_ctas_per_sm(2, c->f32)));

    c->small_fits = true;
    int64_t max_nz = 0;
    for (const SysDesc &d : c->h_desc) {
        const int64_t nz = int64_t(rp[size_t(d.row_off + d.m)]) - rp[size_t(d.row_off)];
        max_nz = std::max(max_nz, nz);
        if (nz > kSmallMaxNnz) c->small_fits = false;
    }
    // AUTO picks the cluster form where it measured faster: systems of at
    // most 65,536 nonzeros (a lone 2,000 x 2,000 system: 16 vs 25 us per
    // update), or enough of them to give every SM a CTA (128 systems of
    // 1,000-4,000 rows: 14 % faster)
    c->small_auto = c->small_fits && (max_nz <= kSmallAutoNnz || int64_t(c->nsys) * 8 >= int64_t(c->nsm));
    // the cluster form keeps whole copies of r and p in each CTA's shared
    // memory when the largest system's (m + n) entries fit
    int64_t max_mn = 0;
    for (const SysDesc &d : c->h_desc) max_mn = std::max<int64_t>(max_mn, int64_t(d.m) + int64_t(d.n));
    const int64_t vec_bytes = (max_mn * (c->f32 ? 4 : 8) + 15) / 16 * 16;
    c->clu_vec_bytes = c->small_fits && vec_bytes > 0 && vec_bytes <= kClusterVecBytes ? int32_t(vec_bytes) : 0;

    // one system with every tile of a side sliced: warp ranges instead of
    // tiles for that side's sweep
    if (nsys == 1) {
        // one partial per CTA: at most as many CTAs as tiles (the partial arrays' size)
        const int gr = std::max(1, std::min(int(c->h_rt.size()), c->nsm * sweep_ctas_per_sm(3, c->f32)));
        const int gc = std::max(1, std::min(int(c->h_ct.size()), c->nsm * sweep_ctas_per_sm(4, c->f32)));
        TRY_ST(upload_warp_ranges(c->h_rt, rsl_ptr, int64_t(gr) * kWarps, &c->d_rwr));
        TRY_ST(upload_warp_ranges(c->h_ct, csl_ptr, int64_t(gc) * kWarps, &c->d_cwr));
        c->rsl.wr = c->d_rwr;
        c->csl.wr = c->d_cwr;
        if (c->d_rwr) c->grid_r = gr;
        if (c->d_cwr) c->grid_c = gc;
        // schedule COOP: one cooperative grid for both sides
        const int per_sm = coop_ctas_per_sm(c->f32);
        if (c->d_rwr && c->d_cwr && per_sm > 0) {
            const int g = c->nsm * per_sm;
            TRY_ST(upload_warp_ranges(c->h_rt, rsl_ptr, int64_t(g) * kWarps, &c->d_coop_rwr));
            TRY_ST(upload_warp_ranges(c->h_ct, csl_ptr, int64_t(g) * kWarps, &c->d_coop_cwr));
            TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_coop_part), 8 * 4 * size_t(g), "partials"));
            TRY_ST(dalloc(reinterpret_cast<void **>(&c->d_coop_bar), 4 * 4, "barrier"));
            if (c->d_coop_rwr && c->d_coop_cwr) c->coop_grid = g;
        }
    }
#undef TRY_ST

    SweepArgs &a = c->args;
    a.row_ptr = c->d_row_ptr;
    a.col_idx = c->d_col_idx;
    a.val = c->d_val;
    a.col_ptr = c->d_col_ptr;
    a.row_idx = c->d_row_idx;
    a.cval = c->d_cval;
    a.rtiles = c->d_rt;
    a.ctiles = c->d_ct;
    a.vtiles = c->d_vt;
    a.n_rtiles = int32_t(c->h_rt.size());
    a.n_ctiles = int32_t(c->h_ct.size());
    a.n_vtiles = int32_t(c->h_vt.size());
    a.desc = c->d_desc;
    a.st = c->d_st;
    a.part_row = c->d_part_row;
    a.part_col = c->d_part_col;
    a.part_upd = c->d_part_upd;
    a.n_active = c->d_active;
    a.b = c->d_b;
    a.x = c->d_x;
    a.r = c->d_r;
    a.p = c->d_p;
    a.u = c->d_u;
    a.w = nullptr;
    a.winv = nullptr;
    a.wf = nullptr;
    a.winvf = nullptr;
    a.rsl = c->rsl;
    a.csl = c->csl;
    *out = c;
    return PLSS_OK;
}

// ---------------------------------------------------------------------------
// The iteration driver: chunks of bodies captured once as CUDA graphs
// ---------------------------------------------------------------------------

static plss_status get_graph(plss_ctx *c, int chunk, bool w_on, bool prof, cudaGraphExec_t *out) {
    const int key = chunk * 4 + (w_on ? 1 : 0) + (prof ? 2 : 0);
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
        *out = it->second;
        return PLSS_OK;
    }
    SweepArgs a = c->args;
    a.w = w_on ? c->d_w : nullptr;
    a.winv = w_on ? c->d_w + c->n : nullptr;
    a.wf = w_on && c->d_wf ? c->d_wf : nullptr;
    a.winvf = w_on && c->d_wf ? c->d_wf + c->n : nullptr;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    while (prof && c->prof_ev.size() < size_t(4 * chunk)) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) {
            e = cudaErrorMemoryAllocation;
            break;
        }
        c->prof_ev.push_back(ev);
    }
    for (int i = 0; i < chunk && e == cudaSuccess; ++i) {
        cudaEvent_t *ev = prof ? &c->prof_ev[size_t(4 * i)] : nullptr;
        if (prof) e = cudaEventRecordWithFlags(ev[0], c->cap_stream, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_col_sweep(a, c->f32, c->grid_c, c->cap_stream);
        if (prof && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[1], c->cap_stream, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_update(a, c->f32, c->grid_v, c->cap_stream);
        if (prof && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2], c->cap_stream, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_row_sweep(a, c->f32, c->grid_r, c->cap_stream);
        if (prof && e == cudaSuccess) e = cudaEventRecordWithFlags(ev[3], c->cap_stream, cudaEventRecordExternal);
    }
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(PLSS_ERR_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        cudaGetLastError();
        return fail(PLSS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e3));
    }
    c->graphs[key] = ge;
    *out = ge;
    return PLSS_OK;
}

plss_status ensure_weights(plss_ctx *c, int32_t w_mode, cudaStream_t s) {
    if (w_mode == PLSS_W_IDENTITY) return PLSS_OK;
    if (w_mode != PLSS_W_COLNORM && w_mode != PLSS_W_COLNORM2)
        return fail(PLSS_ERR_INVALID, "unknown w_mode %d", w_mode);
    if (c->w_mode_cur == w_mode) return PLSS_OK;
    CUDA_TRY(launch_colweights(c->d_col_ptr, c->d_cval, c->f32, c->n, w_mode, c->d_w, c->d_w + c->n,
                               c->d_wf, c->d_wf ? c->d_wf + c->n : nullptr, s));
    c->w_mode_cur = w_mode;
    return PLSS_OK;
}

plss_status check_opts(const plss_opts *o) {
    if (!o) return fail(PLSS_ERR_INVALID, "opts is NULL");
    if (!(o->tol >= 0.0) || !std::isfinite(o->tol)) return fail(PLSS_ERR_INVALID, "tol must be finite and >= 0");
    if (o->hist_cap < 0) return fail(PLSS_ERR_INVALID, "hist_cap < 0");
    if (!(o->inner_tol >= 0.0) || !(o->inner_tol < 1.0)) return fail(PLSS_ERR_INVALID, "inner_tol must be in [0, 1)");
    if (o->hist_cap > 0 && !o->hist) return fail(PLSS_ERR_INVALID, "hist_cap > 0 with hist NULL");
    if (o->profile < 0) return fail(PLSS_ERR_INVALID, "profile < 0");
    if (o->refine_mode != PLSS_REFINE_RESTART && o->refine_mode != PLSS_REFINE_REPLACE)
        return fail(PLSS_ERR_INVALID, "unknown refine_mode %d", o->refine_mode);
    if (o->schedule != PLSS_SCHED_AUTO && o->schedule != PLSS_SCHED_GRID && o->schedule != PLSS_SCHED_SMALL &&
        o->schedule != PLSS_SCHED_COOP)
        return fail(PLSS_ERR_INVALID, "unknown schedule %d", o->schedule);
    return PLSS_OK;
}

// Copies one input vector into the context's device buffer.
plss_status put_vec(double *dst, const double *src, int64_t len, bool dev, cudaStream_t s) {
    if (len == 0) return PLSS_OK;
    if (!src) {
        CUDA_TRY(cudaMemsetAsync(dst, 0, size_t(len) * 8, s));
        return PLSS_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(dst, src, size_t(len) * 8, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return PLSS_OK;
}

plss_status get_vec(double *dst, const double *src, int64_t len, bool dev, cudaStream_t s) {
    if (len == 0 || !dst) return PLSS_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, src, size_t(len) * 8, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return PLSS_OK;
}

// ||b - A x||/||b|| per system, from the context's b and x buffers.
plss_status true_relres(plss_ctx *c, cudaStream_t s, std::vector<double> &rel) {
    CUDA_TRY(launch_spmv(c->d_row_ptr, c->d_col_idx, c->d_val, c->f32, c->d_rt, int32_t(c->h_rt.size()),
                         c->d_x, c->d_vout, c->d_b, c->d_part_res, c->grid_r, s));
    std::vector<double> part(c->h_rt.size());
    CUDA_TRY(cudaMemcpyAsync(part.data(), c->d_part_res, 8 * part.size(), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    rel.assign(size_t(c->nsys), 0.0);
    for (int32_t sy = 0; sy < c->nsys; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        double ss = 0.0;
        for (int32_t t = 0; t < d.rt_count; ++t) ss += part[size_t(d.rt_begin + t)];
        const double nb = c->h_st[sy].nb;
        rel[size_t(sy)] = nb > 0.0 ? std::sqrt(ss) / nb : 0.0;
    }
    return PLSS_OK;
}

// resume: go on from the state the context holds (b, x, r, p, u and the
// per-system scalars of a solve the update cap stopped, or of
// plss_state_load) instead of starting from b and x0.
plss_status run_residual(plss_ctx *c, const double *const *b, const double *const *x0,
                         double *const *xo, const plss_opts *o, plss_result *res, bool resume = false) {
    TraceRange tr(resume ? "plss: resume (residual sketch)" : "plss: solve (residual sketch)");
    plss_status st = check_opts(o);
    if (st != PLSS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(o->stream);
    const bool dev = o->io_device != 0;
    for (int32_t sy = 0; sy < c->nsys && !resume; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        if (d.m > 0 && !b[sy]) return fail(PLSS_ERR_INVALID, "b is NULL (system %d)", sy);
        st = put_vec(c->d_b + d.row_off, b[sy], d.m, dev, s);
        if (st != PLSS_OK) return st;
        st = put_vec(c->d_x + d.col_off, x0 ? x0[sy] : nullptr, d.n, dev, s);
        if (st != PLSS_OK) return st;
    }
    st = ensure_weights(c, o->w_mode, s);
    if (st != PLSS_OK) return st;
    const bool w_on = o->w_mode != PLSS_W_IDENTITY;
    if (o->hist_cap > 0 && o->hist_cap > c->hist_cap_alloc) {
        dfree(c->d_hist);
        c->d_hist = nullptr;
        c->hist_cap_alloc = 0;
        st = dalloc(reinterpret_cast<void **>(&c->d_hist), size_t(o->hist_cap) * 5 * 8, "hist");
        if (st != PLSS_OK) return st;
        c->hist_cap_alloc = o->hist_cap;
    }
    int64_t maxit_all = 0, hist_k0 = 0;
    CUDA_TRY(cudaStreamSynchronize(s));   // h_st may still be read by an earlier copy
    if (resume) {
        if (!c->state_valid) return fail(PLSS_ERR_INVALID, "no residual-sketch state to resume: solve or load one first");
        CUDA_TRY(cudaMemcpy(c->h_st, c->d_st, sizeof(SysState) * size_t(c->nsys), cudaMemcpyDeviceToHost));
        for (int32_t sy = 0; sy < c->nsys; ++sy)
            if (c->h_st[sy].phase != PH_DONE)
                return fail(PLSS_ERR_INVALID, "the state to resume is not that of a finished solve (system %d)", sy);
        int32_t active = 0;
        for (int32_t sy = 0; sy < c->nsys; ++sy) {
            const SysDesc &d = c->h_desc[size_t(sy)];
            SysState &z = c->h_st[sy];
            z.hist = nullptr;
            z.hist_cap = 0;
            if (sy == 0 && o->hist_cap > 0) {
                z.hist = c->d_hist;
                z.hist_cap = o->hist_cap;
            }
            z.tol = o->tol;
            z.maxit = o->maxit < 0 ? int64_t(d.n) : o->maxit;
            if (z.phase == PH_DONE && z.status == PLSS_NOT_CONVERGED && (z.resume & 0x100) && z.iters < z.maxit) {
                // the transition the stopping rule kept when the cap stopped it
                z.phase = z.resume & 0xf;
                if (z.resume & 0x10) z.since = 0;
                if (z.resume & 0x20) z.restart_next = 0;
                z.status = 0;
                z.resume = 0;
                ++active;
            }
            maxit_all = std::max(maxit_all, z.maxit);
        }
        *c->h_active = active;
        hist_k0 = c->h_st[0].iters;
    }
    for (int32_t sy = 0; sy < c->nsys && !resume; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        SysState z;
        std::memset(&z, 0, sizeof z);
        z.tol = o->tol;
        z.maxit = o->maxit < 0 ? int64_t(d.n) : o->maxit;
        const bool replace = o->refine_mode == PLSS_REFINE_REPLACE;
        z.refine = (c->f32 || replace) ? std::max<int64_t>(0, o->refine_period) : 0;
        z.inner_tol2 = c->f32 ? o->inner_tol * o->inner_tol : 0.0;
        z.stop_on_true = (c->f32 || o->stop_on_true) ? 1 : 0;
        z.replace = replace ? 1 : 0;
        z.restart_next = 1;   // the first set-up row sweep begins the recursion
        z.phase = PH_SETUP;
        z.nb = 0.0;
        if (sy == 0 && o->hist_cap > 0) {
            z.hist = c->d_hist;
            z.hist_cap = o->hist_cap;
        }
        c->h_st[sy] = z;
        maxit_all = std::max(maxit_all, z.maxit);
    }
    if (!resume) *c->h_active = c->nsys;
    c->state_valid = true;
    CUDA_TRY(cudaMemcpyAsync(c->d_st, c->h_st, sizeof(SysState) * size_t(c->nsys), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->d_active, c->h_active, 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaEventRecord(c->ev0, s));
    // Every body either applies an update or finishes a system, except
    // restarts (at most one per update), so 2 (maxit + 2) bodies suffice.
    const int64_t body_cap = 2 * (maxit_all + 2) + 8;
    const bool prof = o->profile != 0;
    const int64_t period = std::max<int64_t>(1, o->profile);   // profile one chunk in `period`
    int64_t bodies = 0, nchunk = 0;
    int chunk = 1;
    const bool idle = *c->h_active <= 0;   // a resume with nothing left to do
    const bool small = !idle && (o->schedule == PLSS_SCHED_SMALL ? c->small_fits
                                                                  : (o->schedule == PLSS_SCHED_AUTO && c->small_auto));
    const bool coop = !idle && !small && o->schedule == PLSS_SCHED_COOP && c->coop_grid > 0;
    if (coop) {
        // one system on the whole GPU, whole bodies per cooperative launch
        SweepArgs a = c->args;
        a.w = w_on ? c->d_w : nullptr;
        a.winv = w_on ? c->d_w + c->n : nullptr;
        a.wf = w_on && c->d_wf ? c->d_wf : nullptr;
        a.winvf = w_on && c->d_wf ? c->d_wf + c->n : nullptr;
        int32_t per = 16;
        for (;;) {
            CUDA_TRY(launch_coop_solve(a, c->f32, c->coop_grid, c->d_coop_rwr, c->d_coop_cwr, c->d_coop_part,
                                       c->d_coop_bar, per, s));
            bodies += per;
            uint32_t bar[4] = {0, 0, 0, 0};
            CUDA_TRY(cudaMemcpyAsync(c->h_active, c->d_active, 4, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaMemcpyAsync(bar, c->d_coop_bar, sizeof bar, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (bar[2] != 0) return fail(PLSS_ERR_TIMEOUT, "cooperative schedule: a grid barrier waited longer than 2 s");
            if (*c->h_active <= 0) break;
            if (bodies > body_cap) return fail(PLSS_ERR_TIMEOUT, "iteration driver exceeded %lld bodies", (long long)body_cap);
            per = std::min(per * 4, 4096);
        }
    }
    if (small) {
        // one cluster per system, whole bodies per launch
        SweepArgs a = c->args;
        a.w = w_on ? c->d_w : nullptr;
        a.winv = w_on ? c->d_w + c->n : nullptr;
        a.wf = w_on && c->d_wf ? c->d_wf : nullptr;
        a.winvf = w_on && c->d_wf ? c->d_wf + c->n : nullptr;
        int32_t per = 16;
        for (;;) {
            CUDA_TRY(launch_cluster_solve(a, c->f32, c->nsys, per, c->clu_vec_bytes, s));
            bodies += per;
            CUDA_TRY(cudaMemcpyAsync(c->h_active, c->d_active, 4, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (*c->h_active <= 0) break;
            if (bodies > body_cap) return fail(PLSS_ERR_TIMEOUT, "iteration driver exceeded %lld bodies", (long long)body_cap);
            per = std::min(per * 4, 4096);
        }
    }
    while (!idle && !small && !coop) {
        const bool pchunk = prof && nchunk++ % period == 0;
        cudaGraphExec_t g = nullptr;
        st = get_graph(c, chunk, w_on, pchunk, &g);
        if (st != PLSS_OK) return st;
        CUDA_TRY(cudaGraphLaunch(g, s));
        bodies += chunk;
        CUDA_TRY(cudaMemcpyAsync(c->h_active, c->d_active, 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (prof) c->prof_all += 3 * int64_t(chunk);
        // time only chunks in which some system stayed active throughout
        // (after the set-up body), so that launches returning at once after
        // convergence do not enter the per-launch averages
        if (pchunk && *c->h_active > 0 && bodies > 1) {
            for (int i = 0; i < chunk; ++i) {
                const cudaEvent_t *ev = &c->prof_ev[size_t(4 * i)];
                float t[3] = {0.0f, 0.0f, 0.0f};
                CUDA_TRY(cudaEventElapsedTime(&t[1], ev[0], ev[1]));
                CUDA_TRY(cudaEventElapsedTime(&t[2], ev[1], ev[2]));
                CUDA_TRY(cudaEventElapsedTime(&t[0], ev[2], ev[3]));
                for (int q = 0; q < 3; ++q) {
                    c->prof_ms[q] += double(t[q]);
                    c->prof_n[q] += 1;
                }
            }
        }
        if (*c->h_active <= 0) break;
        if (bodies > body_cap) return fail(PLSS_ERR_TIMEOUT, "iteration driver exceeded %lld bodies", (long long)body_cap);
        chunk = std::min(chunk * 4, kMaxChunk);
    }
    CUDA_TRY(cudaEventRecord(c->ev1, s));
    CUDA_TRY(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(SysState) * size_t(c->nsys), cudaMemcpyDeviceToHost, s));
    for (int32_t sy = 0; sy < c->nsys; ++sy) {
        const SysDesc &d = c->h_desc[size_t(sy)];
        st = get_vec(xo ? xo[sy] : nullptr, c->d_x + d.col_off, d.n, dev, s);
        if (st != PLSS_OK) return st;
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    if (o->hist_cap > 0) {
        // rows [k0, updates) of system 0: a resume leaves the rows before it untouched
        const int64_t k = std::min<int64_t>(o->hist_cap, c->h_st[0].iters);
        if (k > hist_k0)
            CUDA_TRY(cudaMemcpy(o->hist + 5 * hist_k0, c->d_hist + 5 * hist_k0, size_t(k - hist_k0) * 5 * 8,
                                cudaMemcpyDeviceToHost));
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    std::vector<double> rel;
    if (prof) c->prof_all += 1;
    st = true_relres(c, s, rel);
    if (st != PLSS_OK) return st;
    plss_status overall = PLSS_OK;
    for (int32_t sy = 0; sy < c->nsys; ++sy) {
        const SysState &z = c->h_st[sy];
        if (res) {
            res[sy].status = z.status;
            res[sy].reserved = 0;
            res[sy].iters = z.iters;
            res[sy].relres_rec = z.relres_rec;
            res[sy].relres_true = rel[size_t(sy)];
            res[sy].seconds = double(ms) * 1e-3;
        }
        if (overall == PLSS_OK && z.status != PLSS_OK) overall = plss_status(z.status);
    }
    return overall;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the state of a residual-sketch solve is the vectors
// b, x, r, p, u and one SysState per system. The buffer is a header, the
// states (device pointers cleared), then the vectors in device layout.
// ---------------------------------------------------------------------------

struct StateHeader {
    char magic[8];        // "PLSSST01"
    int32_t f32, nsys;
    int64_t m, n, nnz;
    int64_t state_size;   // sizeof(SysState)
};

struct StateLayout {
    int64_t states, b, x, r, p, u, total;   // byte offsets and the total size
};

StateLayout state_layout(const plss_ctx *c) {
    const int64_t sb = c->f32 ? 4 : 8;
    auto up8 = [](int64_t v) { return (v + 7) / 8 * 8; };
    StateLayout L;
    L.states = int64_t(sizeof(StateHeader));
    L.b = up8(L.states + int64_t(sizeof(SysState)) * c->nsys);
    L.x = up8(L.b + 8 * c->m);
    L.r = up8(L.x + 8 * c->n);
    L.p = up8(L.r + sb * c->m);
    L.u = up8(L.p + sb * c->n);
    L.total = up8(L.u + sb * c->n);
    return L;
}

plss_status state_copy(plss_ctx *c, unsigned char *buf, int64_t bytes, bool save) {
    const StateLayout L = state_layout(c);
    // a load checks the header (when there is one) before the size, so that
    // a state of another context is named as such
    const int64_t need = save ? L.total : int64_t(sizeof(StateHeader));
    if (bytes < need) return fail(PLSS_ERR_INVALID, "state buffer of %lld bytes, %lld needed", (long long)bytes,
                                  (long long)L.total);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(PLSS_ERR_CUDA, "cudaSetDevice");
    const int64_t sb = c->f32 ? 4 : 8;
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "PLSSST01", 8);
    h.f32 = c->f32 ? 1 : 0;
    h.nsys = c->nsys;
    h.m = c->m;
    h.n = c->n;
    h.nnz = c->nnz;
    h.state_size = int64_t(sizeof(SysState));
    struct Part {
        int64_t off;
        void *dev;
        int64_t len;
    } parts[] = {{L.b, c->d_b, 8 * c->m}, {L.x, c->d_x, 8 * c->n}, {L.r, c->d_r, sb * c->m},
                 {L.p, c->d_p, sb * c->n}, {L.u, c->d_u, sb * c->n}};
    std::vector<SysState> z(static_cast<size_t>(c->nsys));
    if (save) {
        if (!c->state_valid) return fail(PLSS_ERR_INVALID, "no residual-sketch state to save: solve first");
        CUDA_TRY(cudaDeviceSynchronize());
        CUDA_TRY(cudaMemcpy(z.data(), c->d_st, sizeof(SysState) * z.size(), cudaMemcpyDeviceToHost));
        for (SysState &q : z) {
            q.hist = nullptr;
            q.hist_cap = 0;
        }
        std::memcpy(buf, &h, sizeof h);
        std::memcpy(buf + L.states, z.data(), sizeof(SysState) * z.size());
        for (const Part &p : parts)
            if (p.len > 0) CUDA_TRY(cudaMemcpy(buf + p.off, p.dev, size_t(p.len), cudaMemcpyDeviceToHost));
        return PLSS_OK;
    }
    StateHeader g;
    std::memcpy(&g, buf, sizeof g);
    if (std::memcmp(g.magic, h.magic, 8) != 0 || g.state_size != h.state_size)
        return fail(PLSS_ERR_INVALID, "not a state saved by this library version");
    if (g.f32 != h.f32 || g.nsys != h.nsys || g.m != h.m || g.n != h.n || g.nnz != h.nnz)
        return fail(PLSS_ERR_INVALID, "the state belongs to a context of other sizes or storage "
                    "(saved: %d systems, %lld x %lld, %lld nonzeros, %s)", g.nsys, (long long)g.m, (long long)g.n,
                    (long long)g.nnz, g.f32 ? "FP32" : "FP64");
    if (bytes < L.total) return fail(PLSS_ERR_INVALID, "state buffer of %lld bytes, %lld needed", (long long)bytes,
                                     (long long)L.total);
    std::memcpy(z.data(), buf + L.states, sizeof(SysState) * z.size());
    // the counters index the history rows and the phases select the kernels'
    // work: a saved state is always that of a finished solve, with counts >= 0
    // and a kept transition into one of the three running phases
    for (size_t i = 0; i < z.size(); ++i) {
        const SysState &q = z[i];
        const int32_t next = q.resume & 0xf;
        if (q.phase != PH_DONE || q.iters < 0 || q.maxit < 0 || q.since < 0 || q.refine < 0 ||
            ((q.resume & 0x100) && (next != PH_SETUP && next != PH_FIRST && next != PH_RUN)))
            return fail(PLSS_ERR_INVALID, "the state's scalars of system %d are not those of a finished solve",
                        int(i));
    }
    for (SysState &q : z) {
        q.hist = nullptr;
        q.hist_cap = 0;
        q.cnt_row = q.cnt_col = q.cnt_upd = 0;
    }
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(c->d_st, z.data(), sizeof(SysState) * z.size(), cudaMemcpyHostToDevice));
    for (const Part &p : parts)
        if (p.len > 0) CUDA_TRY(cudaMemcpy(p.dev, buf + p.off, size_t(p.len), cudaMemcpyHostToDevice));
    c->state_valid = true;
    return PLSS_OK;
}

}  // namespace plss

using namespace plss;

// ---------------------------------------------------------------------------
// Exported C ABI
// ---------------------------------------------------------------------------

extern "C" {

void plss_opts_default(plss_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->sketch = PLSS_SKETCH_RESIDUAL;
    o->precision = PLSS_FP64;
    o->w_mode = PLSS_W_IDENTITY;
    o->stop_on_true = 0;
    o->tol = 1e-8;
    o->maxit = -1;
    o->refine_period = 0;
    o->kacz_hist = 0;
    o->seed = 0;
    o->io_device = 0;
    o->symmetric = 0;
    o->stream = nullptr;
    o->hist = nullptr;
    o->hist_cap = 0;
    o->profile = 0;
    o->layout = PLSS_LAYOUT_AUTO;
    o->schedule = PLSS_SCHED_AUTO;
    o->tile_shift = 0;
    o->inner_tol = 1e-4;
    o->refine_mode = PLSS_REFINE_RESTART;
}

plss_status plss_create(const plss_csr *A, const plss_opts *o, plss_ctx **out) {
    clear_error();
    if (!out) return fail(PLSS_ERR_INVALID, "out is NULL");
    return ctx_build(A, 1, o, out);
}

plss_status plss_create_batched(const plss_csr *As, int32_t nsys, const plss_opts *o, plss_ctx **out) {
    clear_error();
    if (!out) return fail(PLSS_ERR_INVALID, "out is NULL");
    return ctx_build(As, nsys, o, out);
}

void plss_destroy(plss_ctx *ctx) { ctx_free(ctx); }

plss_status plss_ctx_info(const plss_ctx *ctx, int32_t *nsys, int64_t *m, int64_t *n, int64_t *nnz) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    if (nsys) *nsys = ctx->nsys;
    if (m) *m = ctx->m;
    if (n) *n = ctx->n;
    if (nnz) *nnz = ctx->nnz;
    return PLSS_OK;
}

plss_status plss_ctx_layout(const plss_ctx *ctx, int64_t out[6]) {
    clear_error();
    if (!ctx || !out) return fail(PLSS_ERR_INVALID, "NULL argument");
    int64_t sr = 0, sc = 0;
    for (const Tile &t : ctx->h_rt) sr += (t.group & kSliced) ? 1 : 0;
    for (const Tile &t : ctx->h_ct) sc += (t.group & kSliced) ? 1 : 0;
    out[0] = int64_t(ctx->h_rt.size());
    out[1] = sr;
    out[2] = int64_t(ctx->h_ct.size());
    out[3] = sc;
    out[4] = ctx->sl_elems[0];
    out[5] = ctx->sl_elems[1];
    return PLSS_OK;
}

plss_status plss_solve(plss_ctx *ctx, const double *b, const double *x0, double *x_out,
                       const plss_opts *o, plss_result *res) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    if (ctx->nsys != 1) return fail(PLSS_ERR_INVALID, "plss_solve needs a single-system context");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    if (o->sketch == PLSS_SKETCH_IDENTITY) return run_identity(ctx, b, x0, x_out, o, res);
    if (o->sketch == PLSS_SKETCH_GENERAL) return run_general(ctx, b, x0, x_out, o, res);
    if (o->sketch != PLSS_SKETCH_RESIDUAL) return fail(PLSS_ERR_INVALID, "unknown sketch %d", o->sketch);
    const double *bb[1] = {b};
    const double *xx[1] = {x0};
    double *oo[1] = {x_out};
    return run_residual(ctx, bb, xx, oo, o, res);
}

plss_status plss_resume(plss_ctx *ctx, double *const *x_out, const plss_opts *o, plss_result *res) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    if (o->sketch != PLSS_SKETCH_RESIDUAL) return fail(PLSS_ERR_INVALID, "only the residual sketch resumes");
    return run_residual(ctx, nullptr, nullptr, x_out, o, res, true);
}

int64_t plss_state_bytes(const plss_ctx *ctx) {
    clear_error();
    if (!ctx) {
        fail(PLSS_ERR_INVALID, "ctx is NULL");
        return -1;
    }
    return state_layout(ctx).total;
}

plss_status plss_state_save(plss_ctx *ctx, void *buf, int64_t bytes) {
    clear_error();
    if (!ctx || !buf) return fail(PLSS_ERR_INVALID, "NULL argument");
    return state_copy(ctx, static_cast<unsigned char *>(buf), bytes, true);
}

plss_status plss_state_load(plss_ctx *ctx, const void *buf, int64_t bytes) {
    clear_error();
    if (!ctx || !buf) return fail(PLSS_ERR_INVALID, "NULL argument");
    return state_copy(ctx, const_cast<unsigned char *>(static_cast<const unsigned char *>(buf)), bytes, false);
}

plss_status plss_solve_batched(plss_ctx *ctx, const double *const *b, const double *const *x0,
                               double *const *x_out, const plss_opts *o, plss_result *res) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    if (!b) return fail(PLSS_ERR_INVALID, "b is NULL");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    if (o->sketch == PLSS_SKETCH_IDENTITY) return run_identity_multi(ctx, b, x0, x_out, o, res);
    if (o->sketch != PLSS_SKETCH_RESIDUAL) return fail(PLSS_ERR_INVALID, "unknown sketch %d", o->sketch);
    return run_residual(ctx, b, x0, x_out, o, res);
}

plss_status plss_spmv(plss_ctx *ctx, int32_t transpose, const double *v, double *out, const plss_opts *o) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    if (ctx->nsys != 1) return fail(PLSS_ERR_INVALID, "plss_spmv needs a single-system context");
    plss_opts od;
    plss_opts_default(&od);
    if (!o) o = &od;
    cudaStream_t s = static_cast<cudaStream_t>(o->stream);
    const bool dev = o->io_device != 0;
    const int64_t lin = transpose ? ctx->m : ctx->n;
    const int64_t lout = transpose ? ctx->n : ctx->m;
    if ((lin > 0 && !v) || (lout > 0 && !out)) return fail(PLSS_ERR_INVALID, "NULL vector");
    plss_status st = put_vec(ctx->d_vin, v, lin, dev, s);
    if (st != PLSS_OK) return st;
    if (transpose) {
        CUDA_TRY(launch_spmv(ctx->d_col_ptr, ctx->d_row_idx, ctx->d_cval, ctx->f32, ctx->d_ct,
                             int32_t(ctx->h_ct.size()), ctx->d_vin, ctx->d_vout, nullptr, nullptr, ctx->grid_c, s));
    } else {
        CUDA_TRY(launch_spmv(ctx->d_row_ptr, ctx->d_col_idx, ctx->d_val, ctx->f32, ctx->d_rt,
                             int32_t(ctx->h_rt.size()), ctx->d_vin, ctx->d_vout, nullptr, nullptr, ctx->grid_r, s));
    }
    st = get_vec(out, ctx->d_vout, lout, dev, s);
    if (st != PLSS_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(s));
    return PLSS_OK;
}

plss_status plss_kernel_times(plss_ctx *ctx, double *ms, int64_t *launches, int32_t reset) {
    clear_error();
    if (!ctx) return fail(PLSS_ERR_INVALID, "ctx is NULL");
    for (int q = 0; q < 3; ++q) {
        if (ms) ms[q] = ctx->prof_ms[q];
        if (launches) launches[q] = ctx->prof_n[q];
    }
    if (launches) launches[3] = ctx->prof_all;
    if (reset) {
        for (int q = 0; q < 3; ++q) {
            ctx->prof_ms[q] = 0.0;
            ctx->prof_n[q] = 0;
        }
        ctx->prof_all = 0;
    }
    return PLSS_OK;
}

const char *plss_last_error(void) { return last_error(); }

}  // extern "C"
