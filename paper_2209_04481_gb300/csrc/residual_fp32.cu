// residual_fp32.cu -- FP32-bulk instantiation of the residual kernels (FP32
// flux arithmetic; FP64 pressure recovery in low-beta cells, FP64 ghost
// vector algebra at the inner boundary, FP64 cross-thread reductions).
//
// Kernel choice for one FP32 residual: the register-staged tiled kernel of
// residual.cuh (default), the cellwise reference kernel, or on request the
// TMA-staged kernel of residual_staged.cuh (grids of whole 8 x 32 blocks and
// 16-byte aligned states; otherwise the tiled kernel runs).
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "residual_launch.cuh"
#include "residual_staged.cuh"

namespace crn {
namespace {

constexpr int kStagedTT = 8, kStagedTP = 32;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr if the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 4D tensor map of an FP32 state U[9][n_r][n_theta][n_phi] (phi innermost)
// whose box is one plane's tt x tp block of all nine variables
bool encode_state_map(CUtensorMap* map, const float* U, const Shape& sh, int tt, int tp) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)sh.np, (cuuint64_t)sh.nt, (cuuint64_t)sh.nr, (cuuint64_t)NV};
  const cuuint64_t strides[3] = {(cuuint64_t)sh.np * 4u, (cuuint64_t)sh.np * (cuuint64_t)sh.nt * 4u,
                                 (cuuint64_t)sh.ncell * 4u};
  const cuuint32_t box[4] = {(cuuint32_t)tp, (cuuint32_t)tt, 1u, (cuuint32_t)NV};
  const cuuint32_t estride[4] = {1u, 1u, 1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(U), dims, strides, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int LIM>
cudaError_t launch_staged_lim(crn_grid* g, const float* U, float* R, double* nu, double* du, cudaStream_t st,
                              const CUtensorMap& map) {
  constexpr int TT = kStagedTT, TP = kStagedTP;
  using D = StagedDims<TT, TP>;
  const Shape sh = g->shape;
  const Reduce red = make_reduce(g, nu, du);
  const int ntiles = (sh.nt / TT) * (sh.np / TP);
  const int kc = g->cfg.kchunk_staged;
  const dim3 grid((unsigned)ntiles, (unsigned)((sh.nr + kc - 1) / kc));
  residual_staged<LIM, TT, TP><<<grid, D::NTH, D::BYTES, st>>>(sh, g->g32.geo, g->ph32, g->br, U, R, red,
                                                                       kc, map);
  return cudaGetLastError();
}

cudaError_t launch_staged(crn_grid* g, const float* U, float* R, double* nu, double* du, cudaStream_t st,
                          const CUtensorMap& map) {
  switch (g->d.limiter) {
    case CRN_LIM_NONE: return launch_staged_lim<0>(g, U, R, nu, du, st, map);
    case CRN_LIM_MINMOD: return launch_staged_lim<1>(g, U, R, nu, du, st, map);
    default: return launch_staged_lim<2>(g, U, R, nu, du, st, map);
  }
}

cudaError_t prepare_staged() {
  constexpr int TT = kStagedTT, TP = kStagedTP;
  const int smem = (int)StagedDims<TT, TP>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(residual_staged<0, TT, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(residual_staged<1, TT, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(residual_staged<2, TT, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

}  // namespace

bool staged_shape_ok(int nt, int np) { return nt % kStagedTT == 0 && np % kStagedTP == 0; }
int staged_tiles(int nt, int np) { return (nt / kStagedTT) * (np / kStagedTP); }
int staged_ctas_per_sm_fp32(int limiter) {
  constexpr int TT = kStagedTT, TP = kStagedTP;
  using D = StagedDims<TT, TP>;
  int n = 0;
  cudaError_t e;
  if (limiter == CRN_LIM_NONE)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_staged<0, TT, TP>, D::NTH, D::BYTES);
  else if (limiter == CRN_LIM_MINMOD)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_staged<1, TT, TP>, D::NTH, D::BYTES);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_staged<2, TT, TP>, D::NTH, D::BYTES);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_residual_fp32(crn_grid* g, const float* U, float* R, double* norms_user,
                                 double* dt_user, cudaStream_t st, int* nlaunch) {
  if (g->cfg.staged && (reinterpret_cast<uintptr_t>(U) & 15u) == 0) {
    CUtensorMap map;
    if (encode_state_map(&map, U, g->shape, kStagedTT, kStagedTP)) {
      *nlaunch = 1;
      g->last_kernel = CRN_KERNEL_STAGED;
      return launch_staged(g, U, R, norms_user, dt_user, st, map);
    }
  }
  g->last_kernel = g->d.kernel == CRN_KERNEL_CELLWISE ? CRN_KERNEL_CELLWISE : CRN_KERNEL_TILED_REGS;
  return launch_residual_t<float>(g, U, R, norms_user, dt_user, st, nlaunch);
}
size_t tiled_smem_fp32() { return tiled_smem_t<float>(); }
cudaError_t prepare_fp32() {
  cudaError_t e = prepare_t<float>();
  if (e == cudaSuccess) e = prepare_staged();
  return e;
}
int tiled_ctas_per_sm_fp32(int limiter) { return tiled_ctas_t<float>(limiter); }
cudaError_t launch_efield_fp32(crn_grid* g, const float* U, double* E, bool volume, cudaStream_t st,
                                int* nl) {
  return efield_t<float>(g, U, E, volume, st, nl);
}
size_t ens_member_bytes_fp32() { return sizeof(EnsMember<float>); }
int ens_member_items(const crn_grid* g, int tile, int kchunk) { return ens_items(g, tile, kchunk); }
int ens_fill_fp32(crn_grid* g, const void* U, void* R, int kchunk, int item0, double* nu, double* du, int tile,
                 void* dst) {
  EnsMember<float>* m = static_cast<EnsMember<float>*>(dst);
  ens_fill_t<float>(g, static_cast<const float*>(U), static_cast<float*>(R), kchunk, item0, nu, du, tile, m);
  return m->nitems;
}
cudaError_t launch_ensemble_fp32(const void* dev, int nmem, int nitems, unsigned int* next, int limiter,
                                  int tile, int nctas, cudaStream_t st) {
  return launch_ensemble_t<float>(static_cast<const EnsMember<float>*>(dev), nmem, nitems, next, limiter, tile, nctas,
                                st);
}
int ensemble_ctas_per_sm_fp32(int limiter, int tile) { return ensemble_ctas_t<float>(limiter, tile); }
}  // namespace crn
