// plss_ctx.h -- the context object behind the opaque plss_ctx handle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <vector>

#include "plss.h"
#include "plss_dev.cuh"
#include "plss_plan.h"

namespace plss {

constexpr int64_t kVecTile = 1024;      // entries per update tile
constexpr int kCtasPerSm = 8;           // resident CTAs per SM assumed for grids
constexpr int kMaxChunk = 64;           // bodies per graph launch (max)
constexpr int64_t kSmallMaxNnz = 1 << 20;       // cluster schedule: nonzeros per system at most
constexpr int64_t kSmallAutoNnz = 1 << 16;      // ... chosen by AUTO up to this size (or for many systems)

struct KaczState;   // identity-sketch buffers (plss_kaczmarz.cu)
struct GeneralState;   // general-sketch buffers (plss_general.cu)
struct RhsState;    // multi-right-hand-side buffers (plss_spmm.cu)

}  // namespace plss

struct plss_ctx {
    int32_t nsys = 0;
    int64_t m = 0, n = 0, nnz = 0;   // totals over the packed systems
    bool f32 = false;
    bool symmetric = false;
    int device = 0;
    int nsm = 1;
    std::vector<plss::SysDesc> h_desc;
    std::vector<plss::Tile> h_rt, h_ct, h_vt;

    // matrix (CSR and its transpose) and schedules
    int32_t *d_row_ptr = nullptr, *d_col_idx = nullptr;
    void *d_val = nullptr;
    int32_t *d_col_ptr = nullptr, *d_row_idx = nullptr;
    void *d_cval = nullptr;
    plss::Tile *d_rt = nullptr, *d_ct = nullptr, *d_vt = nullptr;
    plss::SysDesc *d_desc = nullptr;
    plss::SysState *d_st = nullptr;
    double *d_part_row = nullptr, *d_part_col = nullptr, *d_part_upd = nullptr, *d_part_res = nullptr;
    int32_t *d_active = nullptr;

    // iteration vectors
    double *d_b = nullptr, *d_x = nullptr, *d_w = nullptr;
    float *d_wf = nullptr;   // FP32 storage: float w and 1/w
    void *d_r = nullptr, *d_p = nullptr, *d_u = nullptr;
    double *d_vin = nullptr, *d_vout = nullptr;
    double *d_hist = nullptr;
    int64_t hist_cap_alloc = 0;
    int32_t w_mode_cur = -1;

    plss::SysState *h_st = nullptr;   // pinned
    int32_t *h_active = nullptr;      // pinned

    int grid_r = 1, grid_c = 1, grid_v = 1;
    plss::SweepArgs args{};
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<cudaEvent_t> prof_ev;   // 4 per body of the largest profiled chunk
    double prof_ms[3] = {0.0, 0.0, 0.0};
    int64_t prof_n[3] = {0, 0, 0};
    int64_t prof_all = 0;               // every kernel launched by profiled solves

    plss::Sliced rsl{}, csl{};        // sliced copies (csl aliases rsl when symmetric)
    int64_t sl_elems[2] = {0, 0};     // elements of the sliced row / column copies
    int32_t *d_rwr = nullptr, *d_cwr = nullptr;   // warp ranges (Sliced::wr) or null
    // schedule COOP (one system, both sides sliced throughout): warp ranges
    // for its grid, per-CTA partials and barrier words
    int coop_grid = 0;
    int32_t *d_coop_rwr = nullptr, *d_coop_cwr = nullptr;
    double *d_coop_part = nullptr;
    bool state_valid = false;        // the device holds a residual-sketch state (a solve ran, or a load)
    uint32_t *d_coop_bar = nullptr;
    bool small_fits = false;                      // every system fits the cluster schedule
    bool small_auto = false;                      // ... and AUTO picks it
    int32_t clu_vec_bytes = 0;                    // cluster schedule: shared-memory vector copies (0: none)

    plss::KaczState *kacz = nullptr;
    plss::GeneralState *gen = nullptr;
    plss::RhsState *rhs = nullptr;
};

namespace plss {

// Host copy of one CSR with values in double.
struct HostCsr {
    int64_t m = 0, n = 0, nnz = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col_idx;
    std::vector<double> val;
};

// Copies and validates a caller's CSR (host or device arrays).
plss_status fetch_csr(const plss_csr *A, HostCsr &h);

plss_status fail(plss_status s, const char *fmt, ...);
void clear_error();
const char *last_error();
plss_status dalloc(void **p, size_t bytes, const char *what);
void dfree(void *p);
plss_status put_vec(double *dst, const double *src, int64_t len, bool dev, cudaStream_t s);
plss_status get_vec(double *dst, const double *src, int64_t len, bool dev, cudaStream_t s);
plss_status check_opts(const plss_opts *o);
plss_status ensure_weights(plss_ctx *c, int32_t w_mode, cudaStream_t s);
plss_status true_relres(plss_ctx *c, cudaStream_t s, std::vector<double> &rel);
// Resident CTA slots of the sweeps on this device (plan sizes).
PlanSlots plan_slots(int nsm);

// identity sketch (plss_kaczmarz.cu)
plss_status run_identity(plss_ctx *c, const double *b, const double *x0, double *x_out,
                         const plss_opts *o, plss_result *res);
plss_status run_identity_multi(plss_ctx *c, const double *const *b, const double *const *x0,
                               double *const *xo, const plss_opts *o, plss_result *res);
// general sketch (plss_general.cu)
plss_status run_general(plss_ctx *c, const double *b, const double *x0, double *x_out,
                        const plss_opts *o, plss_result *res);
void free_general(plss_ctx *c);
// per-context state of the other solvers
void free_extra(plss_ctx *c);
void free_rhs(plss_ctx *c);

}  // namespace plss
