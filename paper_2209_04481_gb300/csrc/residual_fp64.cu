// residual_fp64.cu -- plain FP64 instantiation of the residual kernels.
#include "residual_launch.cuh"

namespace crn {
cudaError_t launch_residual_fp64(crn_grid* g, const double* U, double* R, double* norms_user,
                                 double* dt_user, cudaStream_t st, int* nlaunch) {
  g->last_kernel = g->d.kernel == CRN_KERNEL_CELLWISE ? CRN_KERNEL_CELLWISE : CRN_KERNEL_TILED_REGS;
  return launch_residual_t<double>(g, U, R, norms_user, dt_user, st, nlaunch);
}
size_t tiled_smem_fp64() { return tiled_smem_t<double>(); }
cudaError_t prepare_fp64() { return prepare_t<double>(); }
int tiled_ctas_per_sm_fp64(int limiter) { return tiled_ctas_t<double>(limiter); }
cudaError_t launch_efield_fp64(crn_grid* g, const double* U, double* E, bool volume, cudaStream_t st,
                                int* nl) {
  return efield_t<double>(g, U, E, volume, st, nl);
}
size_t ens_member_bytes_fp64() { return sizeof(EnsMember<double>); }
int ens_fill_fp64(crn_grid* g, const void* U, void* R, int kchunk, int item0, double* nu, double* du, int tile,
                 void* dst) {
  EnsMember<double>* m = static_cast<EnsMember<double>*>(dst);
  ens_fill_t<double>(g, static_cast<const double*>(U), static_cast<double*>(R), kchunk, item0, nu, du, tile, m);
  return m->nitems;
}
cudaError_t launch_ensemble_fp64(const void* dev, int nmem, int nitems, unsigned int* next, int limiter,
                                  int tile, int nctas, cudaStream_t st) {
  return launch_ensemble_t<double>(static_cast<const EnsMember<double>*>(dev), nmem, nitems, next, limiter, tile, nctas,
                                st);
}
int ensemble_ctas_per_sm_fp64(int limiter, int tile) { return ensemble_ctas_t<double>(limiter, tile); }
}  // namespace crn
