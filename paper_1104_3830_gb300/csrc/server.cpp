// server.cpp -- placeholder, replaced by the continuous-batching server.
#include "sa_internal.h"
using namespace sa;
extern "C" {
sa_status sa_server_create(sa_server** s, int device, size_t hbm_budget, const sa_scale_opts* opts,
                           int32_t solver_threads) { set_error("server not built"); return SA_E_UNSUPPORTED; }
void sa_server_destroy(sa_server* s) {}
sa_status sa_submit(sa_server* s, const void* host_w, sa_wtype wtype, int32_t n, uint64_t* ticket) { return SA_E_UNSUPPORTED; }
sa_status sa_poll(sa_server* s, uint64_t ticket, sa_result* out) { return SA_E_UNSUPPORTED; }
void sa_result_release(sa_server* s, uint64_t ticket) {}
double sa_server_now(const sa_server* s) { return 0.0; }
}
