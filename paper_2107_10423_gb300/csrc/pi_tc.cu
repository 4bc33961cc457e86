#include "pi_tc.cuh"

namespace gw {
gw_status pi_tc_build(const float*, const double*, int, int, int, const double*, int, float*, int, void**, size_t*,
                      cudaStream_t, bool* used) {
  *used = false;
  return GW_OK;
}
}  // namespace gw
