// plss_extra.cu -- entry points still to be filled in.
#include "plss.h"
#include "plss_ctx.h"

namespace plss {
plss_status run_identity(plss_ctx *, const double *, const double *, double *, const plss_opts *,
                         plss_result *) {
    return fail(PLSS_ERR_INVALID, "identity sketch not available in this build");
}
void free_extra(plss_ctx *) {}
}  // namespace plss

using namespace plss;
extern "C" {
plss_status plss_solve_rhs(plss_ctx *, int32_t, const double *, const double *, double *,
                           const plss_opts *, plss_result *) {
    clear_error();
    return fail(PLSS_ERR_INVALID, "plss_solve_rhs not available in this build");
}
void plss_server_opts_default(plss_server_opts *o) {
    if (o) { o->max_slots = 64; o->max_queue = 4096; o->hbm_budget_bytes = 0; o->precision = 0; o->reserved = 0; }
}
plss_status plss_server_create(const plss_server_opts *, plss_server **out) {
    clear_error();
    if (out) *out = nullptr;
    return fail(PLSS_ERR_INVALID, "server not available in this build");
}
plss_status plss_submit(plss_server *, const plss_csr *, const double *, const double *,
                        const plss_opts *, uint64_t *) { return fail(PLSS_ERR_INVALID, "server not available"); }
plss_status plss_poll(plss_server *, uint64_t, double *, plss_result *) { return fail(PLSS_ERR_INVALID, "server not available"); }
plss_status plss_server_stats(plss_server *, int64_t *, int64_t *, int64_t *, int64_t *) { return fail(PLSS_ERR_INVALID, "server not available"); }
void plss_server_destroy(plss_server *) {}
}
