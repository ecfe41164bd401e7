// Serving loop (continuous batching) -- see fse_server_create in fse.h.
#include "../../include/fse.h"
#include "fse_context.h"

extern "C" {
int fse_server_create(fse_server_t** srv, fse_context_t* ctx, const fse_server_cfg_t* cfg) {
  (void)ctx; (void)cfg;
  if (srv) *srv = nullptr;
  return fse::fail(FSE_EINVAL, "server not available");
}
int fse_submit(fse_server_t*, const fse_job_t*, uint64_t*) { return fse::fail(FSE_EINVAL, "no server"); }
int fse_poll(fse_server_t*, uint64_t, int32_t*) { return fse::fail(FSE_EINVAL, "no server"); }
int fse_wait(fse_server_t*, uint64_t, int32_t, fse_stats_t*) { return fse::fail(FSE_EINVAL, "no server"); }
int32_t fse_server_latencies(fse_server_t*, double*, int32_t) { return 0; }
void fse_server_destroy(fse_server_t*) {}
}
