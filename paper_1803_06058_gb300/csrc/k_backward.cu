// k_backward.cu -- vector-Jacobian product of the LOVE variances.
#include "love_internal.cuh"

namespace love {

love_status backward_tables(love_cache*, const FftPlan*, const void*, int, cudaStream_t) {
  return LOVE_ERR_UNSUPPORTED;
}
love_status backward_launch(love_cache*, int64_t, const void*, const void*, void*, double*, double*, cudaStream_t) {
  return LOVE_ERR_UNSUPPORTED;
}

}  // namespace love
