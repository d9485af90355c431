// residual_launch.cuh -- host launcher of the residual kernels for one
// precision; included by residual_fp64.cu and residual_fp32.cu so that the
// two instantiations compile as separate translation units.
#pragma once

#include "corona_internal.h"
#include "residual.cuh"

namespace crn {

template <class T> struct TileFor;
template <> struct TileFor<double> { static constexpr int TT = 8, TP = 32; };
template <> struct TileFor<float> { static constexpr int TT = 8, TP = 32; };

template <class T> const Geo<T>& geo_of(const crn_grid* g);
template <> inline const Geo<double>& geo_of<double>(const crn_grid* g) { return g->g64.geo; }
template <> inline const Geo<float>& geo_of<float>(const crn_grid* g) { return g->g32.geo; }
template <class T> const Phys<T>& phys_of(const crn_grid* g);
template <> inline const Phys<double>& phys_of<double>(const crn_grid* g) { return g->ph64; }
template <> inline const Phys<float>& phys_of<float>(const crn_grid* g) { return g->ph32; }

inline Reduce make_reduce(crn_grid* g, double* norms_user, double* dt_user) {
  Reduce r;
  r.partials = g->partials;
  r.counter = g->counter;
  r.norms_out = g->stats;
  r.dt_out = g->stats + 9;
  r.norms_user = norms_user;
  r.dt_user = dt_user;
  r.err_flags = g->err_flags;
  r.err_cell = g->err_cell;
  r.log_out = nullptr;
  return r;
}

template <class T, int LIM>
cudaError_t launch_lim(crn_grid* g, const T* U, T* R, double* nu, double* du, cudaStream_t st) {
  const Shape sh = g->shape;
  const Geo<T>& geo = geo_of<T>(g);
  const Phys<T>& ph = phys_of<T>(g);
  const Reduce red = make_reduce(g, nu, du);
  if (g->d.kernel == CRN_KERNEL_CELLWISE) {
    const unsigned nb = (unsigned)((sh.ncell + 255) / 256);
    residual_cellwise<T, LIM><<<nb, 256, 0, st>>>(sh, geo, ph, g->br, U, R, red);
    return cudaGetLastError();
  }
  constexpr int TT = TileFor<T>::TT, TP = TileFor<T>::TP;
  using D = TileDims<TT, TP>;
  const size_t smem = D::template smem_bytes<T>();
  const int ntiles = ((sh.nt + TT - 1) / TT) * ((sh.np + TP - 1) / TP);
  const int kc = g->cfg.kchunk_tiled;
  const int nch = (sh.nr + kc - 1) / kc;
  dim3 grid((unsigned)ntiles, (unsigned)nch);
  residual_tiled<T, LIM, TT, TP><<<grid, D::NT, smem, st>>>(sh, geo, ph, g->br, U, R, red, kc);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_residual_t(crn_grid* g, const T* U, T* R, double* nu, double* du,
                              cudaStream_t st, int* nlaunch) {
  *nlaunch = 1;
  switch (g->d.limiter) {
    case CRN_LIM_NONE: return launch_lim<T, 0>(g, U, R, nu, du, st);
    case CRN_LIM_MINMOD: return launch_lim<T, 1>(g, U, R, nu, du, st);
    default: return launch_lim<T, 2>(g, U, R, nu, du, st);
  }
}

// opt the tiled kernels in to their dynamic shared memory on the current device
template <class T>
cudaError_t prepare_t() {
  constexpr int TT = TileFor<T>::TT, TP = TileFor<T>::TP;
  const int smem = (int)TileDims<TT, TP>::template smem_bytes<T>();
  cudaError_t e;
  e = cudaFuncSetAttribute(residual_tiled<T, 0, TT, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(residual_tiled<T, 1, TT, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(residual_tiled<T, 2, TT, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class T>
int tiled_ctas_t(int limiter) {
  constexpr int TT = TileFor<T>::TT, TP = TileFor<T>::TP;
  const size_t smem = TileDims<TT, TP>::template smem_bytes<T>();
  int n = 0;
  cudaError_t e;
  if (limiter == CRN_LIM_NONE)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_tiled<T, 0, TT, TP>, TT * TP, smem);
  else if (limiter == CRN_LIM_MINMOD)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_tiled<T, 1, TT, TP>, TT * TP, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, residual_tiled<T, 2, TT, TP>, TT * TP, smem);
  return e == cudaSuccess ? n : 0;
}

template <class T>
cudaError_t efield_t(crn_grid* g, const T* U, double* E, bool volume, cudaStream_t st, int* nl) {
  if (volume) {
    const int64_t n = g->shape.ncell;
    const int64_t nb = std::min<int64_t>((n + 255) / 256, (int64_t)g->cfg.num_sms * 8);
    cell_efield_kernel<T><<<(unsigned)nb, 256, 0, st>>>(n, U, E);
  } else {
    const int64_t cs = (int64_t)g->shape.nt * g->shape.np;
    boundary_efield_kernel<T><<<(unsigned)((cs + 127) / 128), 128, 0, st>>>(
        g->shape, geo_of<T>(g), phys_of<T>(g), g->br, U, E);
  }
  *nl = 1;
  return cudaGetLastError();
}

// ---- ensemble: member records and the persistent launch
template <class T>
void ens_fill_t(crn_grid* g, const T* U, T* R, int kchunk, int item0, double* norms_user, double* dt_user,
                int tile, EnsMember<T>* m) {
  const int TT = ens_tt(tile), TP = ens_tp(tile);
  m->sh = g->shape;
  m->g = geo_of<T>(g);
  m->ph = phys_of<T>(g);
  m->Br = g->br;
  m->U = U;
  m->R = R;
  m->red = make_reduce(g, norms_user, dt_user);
  m->kchunk = kchunk;
  m->ntiles = ((g->shape.nt + TT - 1) / TT) * ((g->shape.np + TP - 1) / TP);
  m->nitems = m->ntiles * ((g->shape.nr + kchunk - 1) / kchunk);
  m->item0 = item0;
  m->tile = tile;
}

template <class T, int TT, int TP>
cudaError_t launch_ensemble_shape(const EnsMember<T>* dev, int nmem, int nitems, unsigned int* next, int limiter,
                                  int nctas, cudaStream_t st) {
  const size_t smem = TileDims<TT, TP>::template smem_bytes<T>();
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if (limiter == CRN_LIM_NONE)
    residual_ensemble<T, 0, TT, TP><<<nctas, TT * TP, smem, st>>>(dev, nmem, nitems, next);
  else if (limiter == CRN_LIM_MINMOD)
    residual_ensemble<T, 1, TT, TP><<<nctas, TT * TP, smem, st>>>(dev, nmem, nitems, next);
  else
    residual_ensemble<T, 2, TT, TP><<<nctas, TT * TP, smem, st>>>(dev, nmem, nitems, next);
  return cudaGetLastError();
}

// the persistent launch over the members of one tile shape
template <class T>
cudaError_t launch_ensemble_t(const EnsMember<T>* dev, int nmem, int nitems, unsigned int* next, int limiter,
                              int tile, int nctas, cudaStream_t st) {
  if (tile == 0) return launch_ensemble_shape<T, ens_tt(0), ens_tp(0)>(dev, nmem, nitems, next, limiter, nctas, st);
  return launch_ensemble_shape<T, ens_tt(1), ens_tp(1)>(dev, nmem, nitems, next, limiter, nctas, st);
}

template <class T, int TT, int TP>
int ensemble_ctas_shape(int limiter) {
  const int smem = (int)TileDims<TT, TP>::template smem_bytes<T>();
  auto setup = [&](auto kern) {
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TT * TP, smem) != cudaSuccess) return 0;
    return n;
  };
  if (limiter == CRN_LIM_NONE) return setup(residual_ensemble<T, 0, TT, TP>);
  if (limiter == CRN_LIM_MINMOD) return setup(residual_ensemble<T, 1, TT, TP>);
  return setup(residual_ensemble<T, 2, TT, TP>);
}

// shared-memory opt-in and resident CTAs per SM of one tile shape's kernel
template <class T>
int ensemble_ctas_t(int limiter, int tile) {
  return tile == 0 ? ensemble_ctas_shape<T, ens_tt(0), ens_tp(0)>(limiter)
                   : ensemble_ctas_shape<T, ens_tt(1), ens_tp(1)>(limiter);
}

// work items of one member for a tile shape and radial chunk
inline int ens_items(const crn_grid* g, int tile, int kchunk) {
  const int TT = ens_tt(tile), TP = ens_tp(tile);
  return ((g->shape.nt + TT - 1) / TT) * ((g->shape.np + TP - 1) / TP) * ((g->shape.nr + kchunk - 1) / kchunk);
}

template <class T>
size_t tiled_smem_t() {
  using D = TileDims<TileFor<T>::TT, TileFor<T>::TP>;
  return D::template smem_bytes<T>();
}

}  // namespace crn
