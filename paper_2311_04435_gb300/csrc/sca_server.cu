// Serving loop (continuous batching of SCA solve requests).
#include "sca_internal.h"

extern "C" {
struct sca_server { int dummy; };
sca_status sca_server_create(uint64_t, int32_t, sca_server** out) {
  if (out) *out = nullptr;
  sca::set_error("server not built");
  return SCA_EINVAL;
}
sca_status sca_submit(sca_server*, const sca_params*, const sca_adam*, uint64_t*) { return SCA_EINVAL; }
sca_status sca_poll(sca_server*, uint64_t, double*, double*, int32_t*, double*) { return SCA_EINVAL; }
sca_status sca_request_times(sca_server*, uint64_t, double*, double*, double*, double*) { return SCA_EINVAL; }
void sca_server_destroy(sca_server*) {}
}
