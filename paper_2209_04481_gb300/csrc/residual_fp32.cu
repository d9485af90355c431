// residual_fp32.cu -- FP32-bulk instantiation of the residual kernels (FP32
// flux arithmetic; FP64 pressure recovery in low-beta cells, FP64 ghost
// vector algebra at the inner boundary, FP64 cross-thread reductions).
#include "residual_launch.cuh"

namespace crn {
cudaError_t launch_residual_fp32(crn_grid* g, const float* U, float* R, double* norms_user,
                                 double* dt_user, cudaStream_t st, int* nlaunch) {
  return launch_residual_t<float>(g, U, R, norms_user, dt_user, st, nlaunch);
}
size_t tiled_smem_fp32() { return tiled_smem_t<float>(); }
cudaError_t prepare_fp32() { return prepare_t<float>(); }
int tiled_ctas_per_sm_fp32(int limiter) { return tiled_ctas_t<float>(limiter); }
cudaError_t launch_efield_fp32(crn_grid* g, const float* U, double* E, bool volume, cudaStream_t st,
                                int* nl) {
  return efield_t<float>(g, U, E, volume, st, nl);
}
size_t ens_member_bytes_fp32() { return sizeof(EnsMember<float>); }
int ens_fill_fp32(crn_grid* g, const void* U, void* R, int kchunk, int item0, double* nu, double* du, void* dst) {
  EnsMember<float>* m = static_cast<EnsMember<float>*>(dst);
  ens_fill_t<float>(g, static_cast<const float*>(U), static_cast<float*>(R), kchunk, item0, nu, du, m);
  return m->nitems;
}
cudaError_t launch_ensemble_fp32(const void* dev, int nmem, int nitems, unsigned int* next, int limiter,
                                  int nctas, cudaStream_t st) {
  return launch_ensemble_t<float>(static_cast<const EnsMember<float>*>(dev), nmem, nitems, next, limiter, nctas, st);
}
int ensemble_ctas_per_sm_fp32(int limiter) { return ensemble_ctas_t<float>(limiter); }
}  // namespace crn
