// plss_extra.cu -- entry points still to be filled in.
#include "plss.h"
#include "plss_ctx.h"

using namespace plss;
extern "C" {
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
