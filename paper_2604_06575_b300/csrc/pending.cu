// Entry points whose kernels are not in this build yet report
// POLYLAB_ERR_UNSUPPORTED instead of computing anything.
#include "common.cuh"

namespace polylab {

struct GemmOperand {};

polylab_status build_gemm_operand(polylab_plan*, cudaStream_t) { return POLYLAB_ERR_UNSUPPORTED; }
void free_gemm_operand(GemmOperand* g, cudaStream_t) { delete g; }
polylab_status eval_gemm(const polylab_plan*, const double*, int64_t, int, int, double*, double*, double*,
                         cudaStream_t) {
  return POLYLAB_ERR_UNSUPPORTED;
}
polylab_status affine_stochastic(const polylab_plan*, const double*, int64_t, const polylab_an_opts*, double*,
                                 double*, polylab_an_info*, cudaStream_t) {
  return POLYLAB_ERR_UNSUPPORTED;
}

}  // namespace polylab
