// residual_fp64.cu -- plain FP64 instantiation of the residual kernels.
#include "residual_launch.cuh"

namespace crn {
cudaError_t launch_residual_fp64(crn_grid* g, const double* U, double* R, double* norms_user,
                                 double* dt_user, cudaStream_t st, int* nlaunch) {
  return launch_residual_t<double>(g, U, R, norms_user, dt_user, st, nlaunch);
}
size_t tiled_smem_fp64() { return tiled_smem_t<double>(); }
cudaError_t prepare_fp64() { return prepare_t<double>(); }
int tiled_ctas_per_sm_fp64(int limiter) { return tiled_ctas_t<double>(limiter); }
cudaError_t launch_efield_fp64(crn_grid* g, const double* U, double* E, bool volume, cudaStream_t st,
                                int* nl) {
  return efield_t<double>(g, U, E, volume, st, nl);
}
}  // namespace crn
