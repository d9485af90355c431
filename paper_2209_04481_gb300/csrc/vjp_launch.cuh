// vjp_launch.cuh -- host launcher of the residual VJP for one precision;
// included by vjp_fp64.cu and vjp_fp32.cu.
#pragma once

#include <cstdlib>
#include <cstring>

#include "corona_internal.h"
#include "vjp_tiled.cuh"

namespace crn {

template <class T> const Geo<T>& vgeo(const crn_grid* g);
template <> inline const Geo<double>& vgeo<double>(const crn_grid* g) { return g->g64.geo; }
template <> inline const Geo<float>& vgeo<float>(const crn_grid* g) { return g->g32.geo; }
template <class T> const Phys<T>& vphys(const crn_grid* g);
template <> inline const Phys<double>& vphys<double>(const crn_grid* g) { return g->ph64; }
template <> inline const Phys<float>& vphys<float>(const crn_grid* g) { return g->ph32; }

// Which VJP a grid runs.  FP32-bulk grids: the tiled two-pass VJP of
// vjp_tiled.cuh (issue-bound; its on-chip intermediates replace 864 B/cell of
// face scratch that would not fit in L2 at production sizes).  FP64 grids:
// the face/cell pair of vjp.cuh, which evaluates each face exactly once; on
// the FP64 pipe (1/64 of the FP32 rate) the tiled pass's redundant halo faces
// cost more than its scratch traffic saves.  Grids created with the
// cell-wise reference kernel take the face/cell pair too.  CRN_VJP_KERNEL
// ("tiled" or "faces") overrides the choice.
inline bool vjp_uses_scratch(const crn_grid* g) {
  if (const char* e = std::getenv("CRN_VJP_KERNEL")) {
    if (std::strcmp(e, "tiled") == 0) return false;
    if (std::strcmp(e, "faces") == 0) return true;
  }
  return g->d.kernel == CRN_KERNEL_CELLWISE || g->d.precision == CRN_FP64;
}

inline size_t vjp_scratch_elems(const Shape& s) {
  const size_t cs = (size_t)s.nt * s.np;
  return (size_t)4 * NV * ((size_t)(s.nr + 1) * cs + (size_t)s.nr * (s.nt + 1) * s.np + (size_t)s.nr * cs) +
         (size_t)NV * s.ncell;
}

template <class T, int LIM>
cudaError_t vjp_lim(crn_grid* g, const T* U, const T* Rb, T* Ub, double* Brb, cudaStream_t st,
                    int* nl) {
  const Shape sh = g->shape;
  const size_t cs = (size_t)sh.nt * sh.np;
  T* base = static_cast<T*>(g->vjp_buf);
  VjpBufs<T> b;
  b.cr = base;
  b.ct = b.cr + (size_t)4 * NV * (sh.nr + 1) * cs;
  b.cp = b.ct + (size_t)4 * NV * sh.nr * (sh.nt + 1) * sh.np;
  // FP64: recover the primitives once (each FP64 division is costly); FP32:
  // recovery inside the face pass is cheaper than one more pass over memory
  b.W = sizeof(T) == 8 ? b.cp + (size_t)4 * NV * sh.nr * cs : nullptr;
  if (b.W) vjp_prims<T><<<(unsigned)((sh.ncell + 255) / 256), 256, 0, st>>>(sh, vphys<T>(g), U, b.W);
  const int64_t nf = (int64_t)(sh.nr + 1) * (int64_t)cs + (int64_t)sh.nr * (sh.nt + 1) * sh.np +
                     (int64_t)sh.nr * (int64_t)cs;
  vjp_faces<T, LIM><<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(sh, vgeo<T>(g), vphys<T>(g), g->br, U, Rb, b);
  const unsigned nbc = (unsigned)((sh.ncell + 127) / 128);
  vjp_cells<T><<<nbc, 128, 0, st>>>(sh, vgeo<T>(g), vphys<T>(g), g->br, U, Rb, b, Ub, Brb);
  *nl = b.W ? 3 : 2;
  return cudaGetLastError();
}

// Tile of the lateral pass: FP32 8 x 32 (256 threads, two CTAs per SM),
// FP64 8 x 16 (its shared memory is twice as large per cell).
template <class T> struct LatTile;
template <> struct LatTile<float> { static constexpr int TT = 8, TP = 32, MINB = 2; };
template <> struct LatTile<double> { static constexpr int TT = 8, TP = 16, MINB = 2; };

template <class T, int LIM>
cudaError_t vjp_tiled_lim(crn_grid* g, const T* U, const T* Rb, T* Ub, double* Brb, cudaStream_t st,
                          int* nl) {
  constexpr int TT = LatTile<T>::TT, TP = LatTile<T>::TP;
  using D = LatDims<TT, TP>;
  const Shape sh = g->shape;
  const int64_t cs = (int64_t)sh.nt * sh.np;
  auto krad = vjp_radial<T, LIM>;
  auto klat = vjp_lateral<T, LIM, TT, TP, LatTile<T>::MINB>;
  constexpr size_t smem_rad = radial_smem_bytes<T>();
  constexpr size_t smem_lat = D::template smem_bytes<T>();
  // the shared-memory opt-in, once per instantiation and device
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(krad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rad);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(klat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_lat);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const dim3 grad((unsigned)((cs + RCOL - 1) / RCOL), (unsigned)((sh.nr + RK - 1) / RK));
  krad<<<grad, RF * RCOL, smem_rad, st>>>(sh, vgeo<T>(g), vphys<T>(g), g->br, U, Rb, Ub, Brb);
  const int ntiles = ((sh.nt + TT - 1) / TT) * ((sh.np + TP - 1) / TP);
  klat<<<dim3((unsigned)ntiles, (unsigned)sh.nr), TT * TP, smem_lat, st>>>(sh, vgeo<T>(g), vphys<T>(g), U, Rb,
                                                                             Ub);
  *nl = 2;
  return cudaGetLastError();
}

template <class T>
cudaError_t vjp_t(crn_grid* g, const T* U, const T* Rb, T* Ub, double* Brb, cudaStream_t st, int* nl) {
  // the scratch is sized for the grid's own precision: a VJP in the other
  // precision (the FP64 outer products of an FP32-bulk grid's adjoint) is tiled
  const bool own = (sizeof(T) == 8) == (g->d.precision == CRN_FP64);
  const bool ref = own && vjp_uses_scratch(g);
  switch (g->d.limiter) {
    case CRN_LIM_NONE:
      return ref ? vjp_lim<T, 0>(g, U, Rb, Ub, Brb, st, nl) : vjp_tiled_lim<T, 0>(g, U, Rb, Ub, Brb, st, nl);
    case CRN_LIM_MINMOD:
      return ref ? vjp_lim<T, 1>(g, U, Rb, Ub, Brb, st, nl) : vjp_tiled_lim<T, 1>(g, U, Rb, Ub, Brb, st, nl);
    default:
      return ref ? vjp_lim<T, 2>(g, U, Rb, Ub, Brb, st, nl) : vjp_tiled_lim<T, 2>(g, U, Rb, Ub, Brb, st, nl);
  }
}

}  // namespace crn
