// vjp_fp64.cu -- FP64 instantiation of the residual VJP.
#include "vjp_launch.cuh"

namespace crn {
cudaError_t launch_vjp_fp64(crn_grid* g, const double* U, const double* Rb, double* Ub, double* Brb,
                            cudaStream_t st, int* nl) {
  return vjp_t<double>(g, U, Rb, Ub, Brb, st, nl);
}
size_t vjp_scratch_bytes(const crn_grid* g) {
  if (!vjp_uses_scratch(g)) return 0;
  return vjp_scratch_elems(g->shape) * (g->d.precision == CRN_FP64 ? 8 : 4);
}
}  // namespace crn
