// vjp_fp32.cu -- FP32 instantiation of the residual VJP (the adjoint
// arithmetic in FP32, the inner-ghost adjoint in FP64).
#include "vjp_launch.cuh"

namespace crn {
cudaError_t launch_vjp_fp32(crn_grid* g, const float* U, const float* Rb, float* Ub, double* Brb,
                            cudaStream_t st, int* nl) {
  return vjp_t<float>(g, U, Rb, Ub, Brb, st, nl);
}
}  // namespace crn
