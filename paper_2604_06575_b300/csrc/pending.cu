// Entry points whose kernels are not in this build yet report
// POLYLAB_ERR_UNSUPPORTED instead of computing anything.
#include "common.cuh"

namespace polylab {

polylab_status affine_stochastic(const polylab_plan*, const double*, int64_t, const polylab_an_opts*, double*,
                                 double*, polylab_an_info*, cudaStream_t) {
  return POLYLAB_ERR_UNSUPPORTED;
}

}  // namespace polylab
