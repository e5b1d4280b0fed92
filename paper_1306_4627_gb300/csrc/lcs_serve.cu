// Serving entry points (continuous batching) — placeholder until the scheduler lands.
#include "lcs_ctx.h"

extern "C" int lcs_serve_create(lcs_ctx*, const lcs_serve_cfg*, lcs_server** out) {
  if (out) *out = nullptr;
  return LCS_ERR_INTERNAL;
}
extern "C" int lcs_serve_submit(lcs_server*, const uint8_t*, uint64_t, const uint8_t*, uint64_t, uint32_t, uint64_t*) {
  return LCS_ERR_INVALID;
}
extern "C" int lcs_serve_poll(lcs_server*, uint64_t, lcs_result*) { return LCS_ERR_INVALID; }
extern "C" int lcs_serve_wait(lcs_server*, uint64_t, double, lcs_result*) { return LCS_ERR_INVALID; }
extern "C" void lcs_result_release(lcs_server*, uint64_t) {}
extern "C" void lcs_serve_destroy(lcs_server*) {}
