// tcgen05 (5th-generation tensor core) 3xTF32 rank-nb update for sm_103a.
#include "sca_internal.h"

namespace sca {

bool tc_supported() { return false; }
sca_status tc_prepare(Engine&) { return SCA_OK; }
void tc_release(Engine&) {}
sca_status tc_update(Engine&, int, int, int, int, int, bool, cudaStream_t) {
  set_error("tcgen05 update not available");
  return SCA_EINVAL;
}

}  // namespace sca
