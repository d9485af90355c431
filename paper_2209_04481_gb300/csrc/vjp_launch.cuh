// vjp_launch.cuh -- host launcher of the residual VJP for one precision;
// included by vjp_fp64.cu and vjp_fp32.cu.
#pragma once

#include "corona_internal.h"
#include "vjp.cuh"

namespace crn {

template <class T> const Geo<T>& vgeo(const crn_grid* g);
template <> inline const Geo<double>& vgeo<double>(const crn_grid* g) { return g->g64.geo; }
template <> inline const Geo<float>& vgeo<float>(const crn_grid* g) { return g->g32.geo; }
template <class T> const Phys<T>& vphys(const crn_grid* g);
template <> inline const Phys<double>& vphys<double>(const crn_grid* g) { return g->ph64; }
template <> inline const Phys<float>& vphys<float>(const crn_grid* g) { return g->ph32; }

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

template <class T>
cudaError_t vjp_t(crn_grid* g, const T* U, const T* Rb, T* Ub, double* Brb, cudaStream_t st, int* nl) {
  switch (g->d.limiter) {
    case CRN_LIM_NONE: return vjp_lim<T, 0>(g, U, Rb, Ub, Brb, st, nl);
    case CRN_LIM_MINMOD: return vjp_lim<T, 1>(g, U, Rb, Ub, Brb, st, nl);
    default: return vjp_lim<T, 2>(g, U, Rb, Ub, Brb, st, nl);
  }
}

}  // namespace crn
