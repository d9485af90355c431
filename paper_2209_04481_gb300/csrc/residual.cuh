// residual.cuh -- residual kernels of the MHD + GLM finite-volume operator.
//
// Two kernels evaluate the same operator R = dU/dt (arXiv 2209.04481,
// Sect. 2.1 second-order FV + HDC, Sect. 2.2 equations, Sect. 3.2 inner
// boundary, Sect. 4.1 outer boundary):
//
//  * residual_tiled   -- the production kernel.  A CTA owns a TT x TP block of
//    (theta, phi) columns and marches outwards in r over a chunk of planes.
//    Each plane (cells + a 2-cell theta/phi halo) is loaded once, its
//    primitives recovered once and kept in a 4-plane shared-memory ring; every
//    face flux of the tile is computed once per plane into shared memory and
//    gathered by the two cells it separates (no atomics); the r-face flux is
//    double-buffered across planes.  Residual norms and the step bound are
//    reduced per thread, per warp (shuffles), per CTA, and across CTAs by the
//    last CTA to finish (fixed order, bitwise reproducible).
//  * residual_cellwise -- a deliberately simple reference kernel: one thread
//    per cell re-evaluates all six of its faces from global memory.
#pragma once

#include "mhd_device.cuh"

namespace crn {

// where the reductions and error reports go
struct Reduce {
  double* partials;          // [gridDim.x * gridDim.y][16]
  unsigned int* counter;     // CTA arrival counter, reset by the last CTA
  double* norms_out;         // [9] L2 norms (always written)
  double* dt_out;            // [1] min V / sum lambda |S| (always written)
  double* norms_user;        // optional copy for the caller
  double* dt_user;           // optional copy for the caller
  unsigned int* err_flags;   // bit 0: non-physical or non-finite cell
  unsigned long long* err_cell;  // lowest flagged cell
  double* log_out;           // if set: write log10 of the 9 norms here instead
};

// ---------------------------------------------------------------------------
// accumulators: FP64 directly, or compensated FP32 (Kahan) per thread that is
// promoted to FP64 for the cross-thread reduction
// ---------------------------------------------------------------------------
template <class T> struct Acc;
template <> struct Acc<double> {
  double s[NV];
  __device__ void init() {
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = 0.0;
  }
  __device__ __forceinline__ void add(int v, double x) { s[v] = fma(x, x, s[v]); }
  __device__ double total(int v) const { return s[v]; }
};
template <> struct Acc<float> {
  float s[NV], c[NV];
  __device__ void init() {
#pragma unroll
    for (int v = 0; v < NV; ++v) { s[v] = 0.f; c[v] = 0.f; }
  }
  __device__ __forceinline__ void add(int v, float x) {
    const float y = fmaf(x, x, -c[v]);
    const float t = s[v] + y;
    c[v] = (t - s[v]) - y;
    s[v] = t;
  }
  __device__ double total(int v) const { return (double)s[v] - (double)c[v]; }
};

__device__ __forceinline__ void flag_bad(const Reduce& red, long long cell) {
  atomicOr(red.err_flags, 1u);
  atomicMin(red.err_cell, (unsigned long long)cell);
}

// Block + grid reduction of 9 sums of squares and one minimum.  Every thread
// of every CTA calls it once at the end of the kernel.
// WARP_DONE: the caller has already reduced within each warp (lane 0 holds
// the warp's sums, every lane the warp's minimum).
template <int NTHREADS, bool WARP_DONE = false>
__device__ void reduce_and_finalize_at(const double (&sum)[NV], double dtmin, const Reduce& red,
                                       double* scratch /* >= (NTHREADS/32) * RED_STRIDE doubles */,
                                       int bid, int nblocks) {
  constexpr int NW = NTHREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[NV + 1];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sum[q];
  v[NV] = dtmin;
  if (!WARP_DONE) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
      v[NV] = fmin(v[NV], __shfl_xor_sync(0xffffffffu, v[NV], off));
    }
  }
  __syncthreads();  // scratch may alias buffers still in use
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q <= NV; ++q) scratch[warp * RED_STRIDE + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x <= NV) {
    const int q = threadIdx.x;
    double a = scratch[q];
    for (int w = 1; w < NW; ++w)
      a = (q < NV) ? a + scratch[w * RED_STRIDE + q] : fmin(a, scratch[w * RED_STRIDE + q]);
    red.partials[(size_t)bid * RED_STRIDE + q] = a;
  }
  __shared__ unsigned int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(red.counter, 1u) == (unsigned)(nblocks - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: fixed-order reduction of all partials
  double acc[NV + 1];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  acc[NV] = INFINITY;
  for (int b = threadIdx.x; b < nblocks; b += NTHREADS) {
    const volatile double* p = red.partials + (size_t)b * RED_STRIDE;
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += p[q];
    acc[NV] = fmin(acc[NV], p[NV]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    acc[NV] = fmin(acc[NV], __shfl_xor_sync(0xffffffffu, acc[NV], off));
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q <= NV; ++q) scratch[warp * RED_STRIDE + q] = acc[q];
  }
  __syncthreads();
  if (threadIdx.x <= NV) {
    const int q = threadIdx.x;
    double a = scratch[q];
    for (int w = 1; w < NW; ++w)
      a = (q < NV) ? a + scratch[w * RED_STRIDE + q] : fmin(a, scratch[w * RED_STRIDE + q]);
    if (red.log_out) {
      if (q < NV) red.log_out[q] = log10(sqrt(a));
    } else if (q < NV) {
      const double nrm = sqrt(a);
      red.norms_out[q] = nrm;
      if (red.norms_user) red.norms_user[q] = nrm;
    } else {
      red.dt_out[0] = a;
      if (red.dt_user) red.dt_user[0] = a;
    }
  }
  if (threadIdx.x == 0) *red.counter = 0u;
}

// the same with the block id and count of the launch grid
template <int NTHREADS, bool WARP_DONE = false>
__device__ __forceinline__ void reduce_and_finalize(const double (&sum)[NV], double dtmin, const Reduce& red,
                                                    double* scratch) {
  reduce_and_finalize_at<NTHREADS, WARP_DONE>(sum, dtmin, red, scratch, blockIdx.y * gridDim.x + blockIdx.x,
                                              gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// reference kernel: one thread per cell
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void load_recover(const T* __restrict__ U, int64_t N, int64_t cell,
                                             const Phys<T>& ph, T (&w)[NV]) {
  T u[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = __ldg(U + v * N + cell);
  recover(u, ph, w);
}

template <class T>
__device__ void cell_prim(const Shape& sh, const Geo<T>& g, const Phys<T>& ph,
                          const double* __restrict__ Br, const T* __restrict__ U, int k, int j,
                          int i, T (&w)[NV]) {
  map_column(j, i, sh.nt, sh.np);
  const int64_t col = (int64_t)j * sh.np + i;
  const int64_t plane = (int64_t)sh.nt * sh.np;
  if (k < 0) {
    T wi[NV];
    load_recover(U, sh.ncell, col, ph, wi);
    const int64_t cs = (int64_t)sh.nt * sh.np;
    inner_ghost_at(wi, Br, col, cs, (double)g.rhat[col], (double)g.rhat[cs + col],
                   (double)g.rhat[2 * cs + col], ph, w);
  } else if (k >= sh.nr) {
    T wi[NV];
    load_recover(U, sh.ncell, (int64_t)(sh.nr - 1) * plane + col, ph, wi);
    const int64_t cs = (int64_t)sh.nt * sh.np;
    outer_ghost(wi, g.rhat[col], g.rhat[cs + col], g.rhat[2 * cs + col], ph, w);
  } else {
    load_recover(U, sh.ncell, (int64_t)k * plane + col, ph, w);
  }
}

// face states from a 4-cell stencil ll, l | r, rr; slopes in units per
// distance (im, ip: inverse centre distances of the two cells' neighbours;
// hl: centre-to-face offset of l, hr: of r)
template <int LIM, class T>
__device__ __forceinline__ void face_states(const T (&ll)[NV], const T (&l)[NV], const T (&r)[NV],
                                            const T (&rr)[NV], T im_l, T ip_l, T hl, T im_r,
                                            T ip_r, T hr, T eps, T (&wl)[NV], T (&wr)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T d = r[v] - l[v];
    const T sl = limited_slope<LIM>((l[v] - ll[v]) * im_l, d * ip_l, eps);
    const T sr = limited_slope<LIM>(d * im_r, (rr[v] - r[v]) * ip_r, eps);
    wl[v] = l[v] + sl * hl;
    wr[v] = r[v] - sr * hr;
  }
}

template <class T, int LIM>
__global__ void __launch_bounds__(256)
residual_cellwise(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br,
                  const T* __restrict__ U, T* __restrict__ R, Reduce red) {
  __shared__ double scratch[8 * RED_STRIDE];
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double sq[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sq[v] = 0.0;
  double dtmin = INFINITY;
  if (cell < sh.ncell) {
    const int i = (int)(cell % sh.np);
    const int j = (int)((cell / sh.np) % sh.nt);
    const int k = (int)(cell / ((int64_t)sh.np * sh.nt));
    const int64_t cs = (int64_t)sh.nt * sh.np;
    const int64_t col = (int64_t)j * sh.np + i;
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = (T)0;
    T lam_sum = (T)0;
    T wc[NV];
    cell_prim(sh, g, ph, Br, U, k, j, i, wc);
    const T one = (T)1, half = (T)0.5;
    // ---- r faces: lower (k - 1/2) and upper (k + 1/2)
    for (int side = 0; side < 2; ++side) {
      const int kl = side == 0 ? k - 1 : k;  // lower cell of the face
      T wl[NV], wr[NV];
      if (kl < 0 || kl >= sh.nr - 1) {  // boundary face: first order
        T a[NV], b[NV];
        cell_prim(sh, g, ph, Br, U, kl, j, i, a);
        cell_prim(sh, g, ph, Br, U, kl + 1, j, i, b);
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = a[v]; wr[v] = b[v]; }
      } else {
        T a[NV], b[NV], c[NV], d[NV];
        cell_prim(sh, g, ph, Br, U, kl - 1, j, i, a);
        cell_prim(sh, g, ph, Br, U, kl, j, i, b);
        cell_prim(sh, g, ph, Br, U, kl + 1, j, i, c);
        cell_prim(sh, g, ph, Br, U, kl + 2, j, i, d);
        face_states<LIM>(a, b, c, d, g.inv_dm[kl], g.inv_dp[kl], g.hp[kl], g.inv_dm[kl + 1],
                         g.inv_dp[kl + 1], g.hm[kl + 1], ph.eps, wl, wr);
      }
      const T area = g.ra[kl + 1] * g.ar[j];
      T f[NV], la;
      rusanov(wl, wr, g.nr[col], g.nr[cs + col], g.nr[2 * cs + col], area, ph, f, la);
      const T sgn = side == 0 ? one : -one;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += sgn * f[v];
      lam_sum += la;
    }
    // ---- theta faces
    const int64_t ts = (int64_t)(sh.nt + 1) * sh.np;
    for (int side = 0; side < 2; ++side) {
      const int jf = side == 0 ? j : j + 1;  // face index
      if (jf == 0 || jf == sh.nt) continue;  // pole faces have zero area
      T a[NV], b[NV], c[NV], d[NV], wl[NV], wr[NV];
      cell_prim(sh, g, ph, Br, U, k, jf - 2, i, a);
      cell_prim(sh, g, ph, Br, U, k, jf - 1, i, b);
      cell_prim(sh, g, ph, Br, U, k, jf, i, c);
      cell_prim(sh, g, ph, Br, U, k, jf + 1, i, d);
      face_states<LIM>(a, b, c, d, one, one, half, one, one, half, ph.eps, wl, wr);
      const int64_t fc = (int64_t)jf * sh.np + i;
      const T area = g.rb[k] * g.at[jf];
      T f[NV], la;
      rusanov(wl, wr, g.nth[fc], g.nth[ts + fc], g.nth[2 * ts + fc], area, ph, f, la);
      const T sgn = side == 0 ? one : -one;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += sgn * f[v];
      lam_sum += la;
    }
    // ---- phi faces (periodic)
    for (int side = 0; side < 2; ++side) {
      const int ifc = side == 0 ? i : i + 1;
      T a[NV], b[NV], c[NV], d[NV], wl[NV], wr[NV];
      cell_prim(sh, g, ph, Br, U, k, j, ifc - 2, a);
      cell_prim(sh, g, ph, Br, U, k, j, ifc - 1, b);
      cell_prim(sh, g, ph, Br, U, k, j, ifc, c);
      cell_prim(sh, g, ph, Br, U, k, j, ifc + 1, d);
      face_states<LIM>(a, b, c, d, one, one, half, one, one, half, ph.eps, wl, wr);
      const int iw = ifc % sh.np;
      const T area = g.rb[k] * g.dtheta;
      T f[NV], la;
      rusanov(wl, wr, g.nph[iw], g.nph[sh.np + iw], (T)0, area, ph, f, la);
      const T sgn = side == 0 ? one : -one;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += sgn * f[v];
      lam_sum += la;
    }
    // ---- divide by the volume, gravity source [Sect. 2.2], GLM damping
    const T vol = g.rv[k] * g.av[j];
    const T ivol = one / vol;
    T r[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) r[v] = acc[v] * ivol;
    const T gk = -g.grav[k];
    const T gx = gk * g.rhat[col], gy = gk * g.rhat[cs + col], gz = gk * g.rhat[2 * cs + col];
    const T rho = wc[0];
    r[1] += rho * gx;
    r[2] += rho * gy;
    r[3] += rho * gz;
    r[7] += rho * (wc[1] * gx + wc[2] * gy + wc[3] * gz);
    r[8] -= ph.psi_damp * wc[8];
    double chk = 0.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R[v * sh.ncell + cell] = r[v];
      sq[v] = (double)r[v] * (double)r[v];
      chk += sq[v];
    }
    dtmin = (double)vol / (double)lam_sum;
    if (!(wc[0] > (T)0) || !(wc[7] > (T)0) || !(chk <= 1.7e308)) flag_bad(red, cell);
  }
  reduce_and_finalize<256>(sq, dtmin, red, scratch);
}

// ---------------------------------------------------------------------------
// boundary electric field diagnostic: E = -V_b x B_b of the face-mean state at
// every inner face, in FP64 [Sect. 2.2 E = -V x B; Sect. 3.2]
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128)
boundary_efield_kernel(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br,
                       const T* __restrict__ U, double* __restrict__ E) {
  const int64_t cs = (int64_t)sh.nt * sh.np;
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= cs) return;
  T wi[NV], wg[NV];
  load_recover(U, sh.ncell, col, ph, wi);
  inner_ghost_at(wi, Br, col, cs, (double)g.rhat[col], (double)g.rhat[cs + col],
                 (double)g.rhat[2 * cs + col], ph, wg);
  double v[3], b[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = 0.5 * ((double)wg[1 + c] + (double)wi[1 + c]);
    b[c] = 0.5 * ((double)wg[4 + c] + (double)wi[4 + c]);
  }
  E[col] = -(v[1] * b[2] - v[2] * b[1]);
  E[cs + col] = -(v[2] * b[0] - v[0] * b[2]);
  E[2 * cs + col] = -(v[0] * b[1] - v[1] * b[0]);
}

// cell-centred E = -V x B = -(m x B) / rho of every cell in FP64 (the volume
// field of Sect. 3.1); E[3][ncell], one cell per thread, grid-stride.
template <class T>
__global__ void __launch_bounds__(256)
cell_efield_kernel(int64_t ncell, const T* __restrict__ U, double* __restrict__ E) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += stride) {
    const double rho = (double)U[c];
    const double m0 = (double)U[ncell + c], m1 = (double)U[2 * ncell + c], m2 = (double)U[3 * ncell + c];
    const double b0 = (double)U[4 * ncell + c], b1 = (double)U[5 * ncell + c], b2 = (double)U[6 * ncell + c];
    const double v0 = m0 / rho, v1 = m1 / rho, v2 = m2 / rho;
    E[c] = -(v1 * b2 - v2 * b1);
    E[ncell + c] = -(v2 * b0 - v0 * b2);
    E[2 * ncell + c] = -(v0 * b1 - v1 * b0);
  }
}

// ---------------------------------------------------------------------------
// production kernel: radial marching over a (theta, phi) tile
// ---------------------------------------------------------------------------
// Thread (jj, ii) owns column (j0 + jj, i0 + ii) of the tile.  Per plane k:
//   A  the prefetched plane k + 2 (own cell + at most one halo cell per thread)
//      is recovered to primitives and stored in a 3-plane ring (k, k+1, k+2)
//   B  the loads of plane k + 3 are issued (they complete during B-E); every
//      cell of plane k gets its theta and phi slopes once, stored as the lower
//      and upper face values; the own column gets the r slope of plane k + 1
//      (registers)
//   C  every theta and phi face of plane k is evaluated once (Rusanov + GLM)
//      into shared memory; the r face k + 1/2 stays in registers
//   E  each cell gathers its six faces, adds gravity and writes R
// The r face k - 1/2 and the upper r face value of plane k + 1 are carried in
// registers from one plane to the next.
template <int TT, int TP>
struct TileDims {
  static constexpr int NT = TT * TP;                            // threads = own columns
  static constexpr int HT = TT + 4, HP = TP + 4, HC = HT * HP;  // halo'd plane
  static constexpr int NHALO = HC - NT;                         // halo positions
  static constexpr int NTV = (TT + 1) * TP;                     // theta faces (rows 0..TT)
  static constexpr int NPV = TT * (TP + 1);                     // phi faces (cols 0..TP)
  static constexpr int NF = NV + 1;                             // 9 fluxes + lambda |S|
  static constexpr int NEXTRA_V = 2 * TP + 2 * TT;              // halo cells needing face values
  static constexpr int NEXTRA_F = TP + TT;                      // faces beyond the own lower faces
  // per-CTA geometry staged once: theta-face normals, phi-face normals, own
  // r-face normals, own radial unit vectors, theta factors of the areas/volumes
  static constexpr int NGEO = 3 * NTV + 2 * (TP + 1) + 6 * NT + (TT + 1) + 2 * TT;
  template <class T>
  static constexpr size_t smem_bytes() {
    return sizeof(T) * ((size_t)3 * NV * HC + (size_t)2 * NV * (NTV + NPV) + (size_t)NGEO);
  }
  // halo position h in [0, NHALO) -> halo'd (row, col)
  __device__ static void halo_rc(int h, int& row, int& col) {
    if (h < 2 * HP) { row = h / HP; col = h % HP; }
    else if (h < 4 * HP) { h -= 2 * HP; row = TT + 2 + h / HP; col = h % HP; }
    else { h -= 4 * HP; row = 2 + h / 4; const int c = h % 4; col = c < 2 ? c : TP + c; }
  }
};

template <class T>
__device__ __forceinline__ void load_raw(const T* __restrict__ src, int64_t N, int64_t c, T (&u)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = __ldg(src + v * N + c);
}

// resident CTAs per SM the register allocation is sized for: two FP32 CTAs
// (16 warps); FP64 CTAs are limited to one by their shared memory anyway
template <class T> struct MinCtas { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };

// One work item of the tiled residual: tile `tile` (row-major over the
// (theta, phi) tiles) and radial chunk `chunk` of one grid; `bid` / `nblocks`
// number the items of that grid for its cross-CTA reduction.
template <class T, int LIM, int TT, int TP>
__device__ __forceinline__ void tiled_item(const Shape& sh, const Geo<T>& g, const Phys<T>& ph,
                                           const double* __restrict__ Br, const T* __restrict__ U,
                                           T* __restrict__ R, const Reduce& red, int kchunk, int tile,
                                           int chunk, int bid, int nblocks, unsigned char* smem_raw) {
  using D = TileDims<TT, TP>;
  constexpr int NT = D::NT, HP = D::HP, HC = D::HC, NTV = D::NTV, NPV = D::NPV, NF = D::NF;
  static_assert(D::NHALO <= NT, "each thread stores at most one halo position");
  static_assert(D::NEXTRA_F <= NT && NT % 32 == 0, "tile shape");
  T* ring = reinterpret_cast<T*>(smem_raw);  // [3][NV][HC]   primitives of planes k..k+2
  T* tvu = ring + 3 * NV * HC;               // [NV][NTV]     theta: upper value of the row below face f
  T* tvl = tvu + NV * NTV;                   // [NV][NTV]     theta: lower value of the row above face f
  T* pvu = tvl + NV * NTV;                   // [NV][NPV]     phi: upper value of the col left of face f
  T* pvl = pvu + NV * NPV;                   // [NV][NPV]     phi: lower value of the col right of face f
  // face fluxes x area overwrite the face values they were computed from (each
  // face is read and written by one thread): flux v of theta face f in
  // tvu[v][f], its lambda x area in tvl[0][f]; likewise phi faces in pvu / pvl
  T* ftb = tvu;
  T* fpb = pvu;
  T* ftl = tvl;                              // lambda x area of theta faces
  T* fpl = pvl;                              // lambda x area of phi faces
  T* gs = pvl + NV * NPV;                    // per-CTA geometry
  T* s_nth = gs;                             // [3][NTV]
  T* s_nph = s_nth + 3 * NTV;                // [2][TP + 1]
  T* s_nr = s_nph + 2 * (TP + 1);            // [3][NT]
  T* s_rh = s_nr + 3 * NT;                   // [3][NT]
  T* s_at = s_rh + 3 * NT;                   // [TT + 1]
  T* s_ar = s_at + (TT + 1);                 // [TT]
  T* s_av = s_ar + TT;                       // [TT]

  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t N = sh.ncell, cs = (int64_t)nt * np;
  const int tid = threadIdx.x;
  const int ntp = (np + TP - 1) / TP;
  const int j0 = (tile / ntp) * TT, i0 = (tile % ntp) * TP;
  const int k0 = chunk * kchunk;
  const int k1 = min(nr, k0 + kchunk);
  const int jj = tid / TP, ii = tid % TP;
  const int jo = j0 + jj, io = i0 + ii;
  const bool own = jo < nt && io < np;
  const int hown = (jj + 2) * HP + (ii + 2);
  // global column of the own position and of this thread's halo position
  int64_t c_own, c_halo = 0;
  int h_halo = -1;
  {
    int j = jo, i = io;
    map_column(j, i, nt, np);
    c_own = (int64_t)j * np + i;
    if (tid < D::NHALO) {
      int row, col;
      D::halo_rc(tid, row, col);
      h_halo = row * HP + col;
      int jh = j0 - 2 + row, ih = i0 - 2 + col;
      map_column(jh, ih, nt, np);
      c_halo = (int64_t)jh * np + ih;
    }
  }
  const int64_t ocol = own ? (int64_t)jo * np + io : 0;
  const T one = (T)1, half = (T)0.5;
  {
    const int64_t ts = (int64_t)(nt + 1) * np;
    for (int q = tid; q < NTV; q += NT) {
      const int f = q / TP, col = q % TP;
      const int jf = min(j0 + f, nt), ic = min(i0 + col, np - 1);
      const int64_t fc = (int64_t)jf * np + ic;
      s_nth[q] = g.nth[fc];
      s_nth[NTV + q] = g.nth[ts + fc];
      s_nth[2 * NTV + q] = g.nth[2 * ts + fc];
    }
    for (int q = tid; q <= TP; q += NT) {
      int ic = i0 + q;
      ic = ic >= np ? ic - np : ic;
      s_nph[q] = g.nph[ic];
      s_nph[TP + 1 + q] = g.nph[np + ic];
    }
    s_nr[tid] = g.nr[ocol];
    s_nr[NT + tid] = g.nr[cs + ocol];
    s_nr[2 * NT + tid] = g.nr[2 * cs + ocol];
    s_rh[tid] = g.rhat[c_own];
    s_rh[NT + tid] = g.rhat[cs + c_own];
    s_rh[2 * NT + tid] = g.rhat[2 * cs + c_own];
    if (tid <= TT) s_at[tid] = g.at[min(j0 + tid, nt)];
    if (tid < TT) {
      s_ar[tid] = g.ar[min(j0 + tid, nt - 1)];
      s_av[tid] = g.av[min(j0 + tid, nt - 1)];
    }
  }

  auto slot = [&](int p) -> T* { return ring + ((p + 3) % 3) * (NV * HC); };

  // raw state of the prefetched plane (own position, halo position)
  T pf_own[NV], pf_halo[NV];
  auto prefetch = [&](int p) {
    const T* src = U + (int64_t)p * cs;
    load_raw(src, N, c_own, pf_own);
    if (h_halo >= 0) load_raw(src, N, c_halo, pf_halo);
  };
  auto store_prefetched = [&](int p) {
    T* dst = slot(p);
    T w[NV];
    recover(pf_own, ph, w);
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[v * HC + hown] = w[v];
    if (h_halo >= 0) {
      recover(pf_halo, ph, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + h_halo] = w[v];
    }
  };
  // outer ghost plane nr from plane nr - 1, own and halo positions
  auto outer_plane = [&]() {
    const T* src = slot(nr - 1);
    T* dst = slot(nr);
    for (int pass = 0; pass < 2; ++pass) {
      const int h = pass == 0 ? hown : h_halo;
      if (h < 0) continue;
      const int64_t c = pass == 0 ? c_own : c_halo;
      T wi[NV], wg[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wi[v] = src[v * HC + h];
      outer_ghost(wi, g.rhat[c], g.rhat[cs + c], g.rhat[2 * cs + c], ph, wg);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + h] = wg[v];
    }
  };
  auto read_own = [&](const T* pl, T (&w)[NV]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = pl[v * HC + hown];
  };
  // r slope of plane p for the own column from planes p-1, p, p+1
  auto r_values = [&](int p, const T (&wm)[NV], const T (&w0)[NV], const T (&wp)[NV], T (&lo)[NV],
                      T (&up)[NV]) {
    const T im = g.inv_dm[p], ip = g.inv_dp[p], hm = g.hm[p], hp = g.hp[p];
    constexpr int VSTEP = sizeof(T) == 8 ? 2 : 1;  // FP64: slopes in pairs
#pragma unroll
    for (int v = 0; v < NV; v += VSTEP) {
      if (VSTEP == 2 && v + 1 < NV) {
        T s, s1;
        limited_slope2<LIM>((w0[v] - wm[v]) * im, (wp[v] - w0[v]) * ip, (w0[v + 1] - wm[v + 1]) * im,
                            (wp[v + 1] - w0[v + 1]) * ip, ph.eps, s, s1);
        lo[v] = fmat(-s, hm, w0[v]);
        up[v] = fmat(s, hp, w0[v]);
        lo[v + 1] = fmat(-s1, hm, w0[v + 1]);
        up[v + 1] = fmat(s1, hp, w0[v + 1]);
      } else {
        const T s = limited_slope<LIM>((w0[v] - wm[v]) * im, (wp[v] - w0[v]) * ip, ph.eps);
        lo[v] = fmat(-s, hm, w0[v]);
        up[v] = fmat(s, hp, w0[v]);
      }
    }
  };

  // ---------------- preamble
  T rL[NV];          // L state of r face k + 1/2 (upper r value of plane k)
  T frl[NF];         // flux x area of r face k - 1/2, lambda x area last
  {
    // own column of planes k0 - 1 and k0 - 2 (loads issued first so that they
    // overlap with those of planes k0 and k0 + 1)
    const int64_t ccol = c_own;
    T um1[NV], um2[NV];
    if (k0 >= 1) load_raw(U + (int64_t)(k0 - 1) * cs, N, ccol, um1);
    if (k0 >= 2) load_raw(U + (int64_t)(k0 - 2) * cs, N, ccol, um2);
    // planes k0 and k0 + 1 into the ring
    for (int p = k0; p <= min(k0 + 1, nr - 1); ++p) {
      prefetch(p);
      store_prefetched(p);
    }
    __syncthreads();
    if (k0 + 1 >= nr) outer_plane();
    __syncthreads();
    T w0[NV], w1[NV], wm1[NV], wm2[NV];
    read_own(slot(k0), w0);
    read_own(slot(k0 + 1), w1);
    // inner ghost for plane -1
    if (k0 >= 1) {
      recover(um1, ph, wm1);
    } else {
      inner_ghost_at(w0, Br, ccol, cs, (double)g.rhat[ccol], (double)g.rhat[cs + ccol],
                     (double)g.rhat[2 * cs + ccol], ph, wm1);
    }
    if (k0 >= 2) {
      recover(um2, ph, wm2);
    } else if (k0 == 1) {
      T wz[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wz[v] = wm1[v];  // plane 0
      inner_ghost_at(wz, Br, ccol, cs, (double)g.rhat[ccol], (double)g.rhat[cs + ccol],
                     (double)g.rhat[2 * cs + ccol], ph, wm2);
    }
    // r face k0 - 1/2
    T wl[NV], wr[NV], up0[NV];
    r_values(k0, wm1, w0, w1, wr, up0);  // lower / upper r values of plane k0
    if (k0 == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) { wl[v] = wm1[v]; wr[v] = w0[v]; }  // boundary: first order
    } else {
      T lo[NV];
      r_values(k0 - 1, wm2, wm1, w0, lo, wl);
    }
    if (own) {
      T f[NV], la;
      const T area = g.ra[k0] * s_ar[jj];
      rusanov(wl, wr, s_nr[tid], s_nr[NT + tid], s_nr[2 * NT + tid], area, ph, f, la);
#pragma unroll
      for (int v = 0; v < NV; ++v) frl[v] = f[v];
      frl[NV] = la;
    } else {
#pragma unroll
      for (int v = 0; v < NF; ++v) frl[v] = (T)0;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) rL[v] = up0[v];
    if (k0 + 2 < nr) prefetch(k0 + 2);
  }

  T sq[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sq[v] = (T)0;
  T dtm = (T)INFINITY;

  for (int k = k0; k < k1; ++k) {
    // ---- A: plane k + 2 enters the ring
    if (k + 2 < nr) store_prefetched(k + 2);
    __syncthreads();
    if (k + 2 == nr) {
      outer_plane();
      __syncthreads();
    }
    // ---- B: prefetch plane k + 3; face values of plane k; r values of plane k + 1
    if (k + 3 < nr) prefetch(k + 3);
    const T* Pk = slot(k);
    T wc[NV];
    read_own(Pk, wc);
    {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* q = Pk + v * HC + hown;
        T st, sp;
        if constexpr (sizeof(T) == 8) {
          limited_slope2<LIM>(wc[v] - q[-HP], q[HP] - wc[v], wc[v] - q[-1], q[1] - wc[v], ph.eps, st, sp);
        } else {
          st = limited_slope<LIM>(wc[v] - q[-HP], q[HP] - wc[v], ph.eps);
          sp = limited_slope<LIM>(wc[v] - q[-1], q[1] - wc[v], ph.eps);
        }
        // explicit FMAs: the same rounding in every kernel inlining this
        tvl[v * NTV + jj * TP + ii] = fmat(-half, st, wc[v]);
        tvu[v * NTV + (jj + 1) * TP + ii] = fmat(half, st, wc[v]);
        pvl[v * NPV + jj * (TP + 1) + ii] = fmat(-half, sp, wc[v]);
        pvu[v * NPV + jj * (TP + 1) + ii + 1] = fmat(half, sp, wc[v]);
      }
      // halo cells whose face values the tile's boundary faces need
      for (int e = tid; e < D::NEXTRA_V; e += NT) {
        int hrow, hcol, dstep, idx;
        T* dst;
        if (e < TP) {                 // theta row -1: upper value -> face 0
          hrow = 1; hcol = e + 2; dstep = HP; dst = tvu; idx = e;
        } else if (e < 2 * TP) {      // theta row TT: lower value -> face TT
          hrow = TT + 2; hcol = e - TP + 2; dstep = HP; dst = tvl; idx = TT * TP + (e - TP);
        } else if (e < 2 * TP + TT) { // phi col -1 of row r: upper value -> face 0
          const int r = e - 2 * TP;
          hrow = r + 2; hcol = 1; dstep = 1; dst = pvu; idx = r * (TP + 1);
        } else {                      // phi col TP of row r: lower value -> face TP
          const int r = e - 2 * TP - TT;
          hrow = r + 2; hcol = TP + 2; dstep = 1; dst = pvl; idx = r * (TP + 1) + TP;
        }
        const bool upper = (dst == tvu) || (dst == pvu);
        const int nstride = (dst == tvu || dst == tvl) ? NTV : NPV;
        constexpr int VSTEP = sizeof(T) == 8 ? 2 : 1;  // FP64: slopes in pairs
#pragma unroll
        for (int v = 0; v < NV; v += VSTEP) {
          const T* q = Pk + v * HC + hrow * HP + hcol;
          const T w = q[0];
          if (VSTEP == 2 && v + 1 < NV) {
            const T* q1 = q + HC;
            const T w1 = q1[0];
            T s, s1;
            limited_slope2<LIM>(w - q[-dstep], q[dstep] - w, w1 - q1[-dstep], q1[dstep] - w1, ph.eps, s, s1);
            dst[v * nstride + idx] = fmat(upper ? half : -half, s, w);
            dst[(v + 1) * nstride + idx] = fmat(upper ? half : -half, s1, w1);
          } else {
            const T s = limited_slope<LIM>(w - q[-dstep], q[dstep] - w, ph.eps);
            dst[v * nstride + idx] = fmat(upper ? half : -half, s, w);
          }
        }
      }
    }
    T rR[NV], rLn[NV];
    if (k + 1 < nr) {
      T w1[NV], w2[NV];
      read_own(slot(k + 1), w1);
      read_own(slot(k + 2), w2);
      r_values(k + 1, wc, w1, w2, rR, rLn);
    }
    __syncthreads();
    // ---- C: faces of plane k
    {
      const T rbk = g.rb[k];
      auto theta_face = [&](int q) {
        const int f = q / TP, col = q % TP;
        const int jf = j0 + f, ic = i0 + col;
        if (jf <= 0 || jf >= nt || ic >= np) {  // poles, ragged rows / columns
#pragma unroll
          for (int v = 0; v < NV; ++v) ftb[v * NTV + q] = (T)0;
          ftl[q] = (T)0;
          return;
        }
        T wl[NV], wr[NV], fl[NV], la;
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = tvu[v * NTV + q]; wr[v] = tvl[v * NTV + q]; }
        rusanov(wl, wr, s_nth[q], s_nth[NTV + q], s_nth[2 * NTV + q], rbk * s_at[f], ph, fl, la);
#pragma unroll
        for (int v = 0; v < NV; ++v) ftb[v * NTV + q] = fl[v];
        ftl[q] = la;
      };
      auto phi_face = [&](int row, int f) {
        const int qq = row * (TP + 1) + f;
        const int jr = j0 + row, ifc = i0 + f;
        if (jr >= nt || ifc > np || (f == TP && ifc - 1 >= np)) {
#pragma unroll
          for (int v = 0; v < NV; ++v) fpb[v * NPV + qq] = (T)0;
          fpl[qq] = (T)0;
          return;
        }
        T wl[NV], wr[NV], fl[NV], la;
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = pvu[v * NPV + qq]; wr[v] = pvl[v * NPV + qq]; }
        rusanov(wl, wr, s_nph[f], s_nph[TP + 1 + f], (T)0, rbk * g.dtheta, ph, fl, la);
#pragma unroll
        for (int v = 0; v < NV; ++v) fpb[v * NPV + qq] = fl[v];
        fpl[qq] = la;
      };
      theta_face(tid);                      // own lower theta face (row jj)
      phi_face(jj, ii);                     // own lower phi face (col ii)
      if (tid < TP) theta_face(NT + tid);   // faces of row TT: warp 0
      if (tid >= 32 && tid < 32 + TT) phi_face(tid - 32, TP);  // faces of col TP: warp 1
    }
    // r face k + 1/2 (own column, registers)
    T fru[NF];
    if (own) {
      T wl[NV], wr[NV], fl[NV], la;
      if (k + 1 < nr) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = rL[v]; wr[v] = rR[v]; }
      } else {  // outer boundary face: first order, interior | ghost
        const T* pg = slot(nr);
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = wc[v]; wr[v] = pg[v * HC + hown]; }
      }
      rusanov(wl, wr, s_nr[tid], s_nr[NT + tid], s_nr[2 * NT + tid], g.ra[k + 1] * s_ar[jj], ph,
              fl, la);
#pragma unroll
      for (int v = 0; v < NV; ++v) fru[v] = fl[v];
      fru[NV] = la;
    }
    __syncthreads();
    // ---- E: gather the six faces of cell (k, jo, io)
    if (own) {
      const int tl = jj * TP + ii, tu = tl + TP;
      const int pl = jj * (TP + 1) + ii, pu = pl + 1;
      T r[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        r[v] = (frl[v] - fru[v]) + (ftb[v * NTV + tl] - ftb[v * NTV + tu]) +
               (fpb[v * NPV + pl] - fpb[v * NPV + pu]);
      const T lam = (frl[NV] + fru[NV]) + (ftl[tl] + ftl[tu]) + (fpl[pl] + fpl[pu]);
      const T vol = g.rv[k] * s_av[jj];
      const T ivol = one / vol;
#pragma unroll
      for (int v = 0; v < NV; ++v) r[v] *= ivol;
      const T gk = -g.grav[k];
      const T gx = gk * s_rh[tid], gy = gk * s_rh[NT + tid], gz = gk * s_rh[2 * NT + tid];
      r[1] += wc[0] * gx;
      r[2] += wc[0] * gy;
      r[3] += wc[0] * gz;
      r[7] += wc[0] * (wc[1] * gx + wc[2] * gy + wc[3] * gz);
      r[8] -= ph.psi_damp * wc[8];
      const int64_t cell = (int64_t)k * cs + ocol;
      T chk = (T)0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R[v * N + cell] = r[v];
        sq[v] = fmat(r[v], r[v], sq[v]);
        chk = fmat(r[v], r[v], chk);
      }
      const T dtc = vol / lam;
      dtm = dtc < dtm ? dtc : dtm;
      if (!(wc[0] > (T)0) || !(wc[7] > (T)0) || !(fabs(chk) < (T)INFINITY)) flag_bad(red, cell);
#pragma unroll
      for (int v = 0; v < NF; ++v) frl[v] = fru[v];
#pragma unroll
      for (int v = 0; v < NV; ++v) rL[v] = rLn[v];
    }
  }
  // ---------------- reductions: warp tree in T, then FP64 across warps and CTAs
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sq[v] += __shfl_xor_sync(0xffffffffu, sq[v], off);
    const T o = __shfl_xor_sync(0xffffffffu, dtm, off);
    dtm = o < dtm ? o : dtm;
  }
  double tot[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = (threadIdx.x & 31) == 0 ? (double)sq[v] : 0.0;
  double* scratch = reinterpret_cast<double*>(smem_raw);
  reduce_and_finalize_at<NT, true>(tot, (double)dtm, red, scratch, bid, nblocks);
}

// one grid: block (x, y) = (tile, radial chunk)
template <class T, int LIM, int TT, int TP>
__global__ void __launch_bounds__(TT * TP, MinCtas<T>::value)
residual_tiled(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br,
               const T* __restrict__ U, T* __restrict__ R, Reduce red, int kchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tiled_item<T, LIM, TT, TP>(sh, g, ph, Br, U, R, red, kchunk, blockIdx.x, blockIdx.y,
                             blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y, smem_raw);
}

// ---------------------------------------------------------------------------
// ensemble: many grids (same precision and limiter, any sizes) in one
// persistent launch.  Work items are (member, tile, radial chunk), numbered
// member by member; CTAs take items from a global counter (zeroed before the
// launch) until none are left.  Each member keeps its own reduction scratch,
// so its norms and dtmin come out exactly as from its own launch with the
// same radial chunk.  The kernel is instantiated per (theta, phi) tile shape;
// members with another shape go to that shape's launch.
// ---------------------------------------------------------------------------

template <class T>
struct EnsMember {
  Shape sh;
  Geo<T> g;
  Phys<T> ph;
  const double* Br;
  const T* U;
  T* R;
  Reduce red;
  int kchunk, ntiles, nitems, item0, tile;
};


template <class T, int LIM, int TT, int TP>
__global__ void __launch_bounds__(TT * TP, MinCtas<T>::value)
residual_ensemble(const EnsMember<T>* __restrict__ mem, int nmem, int nitems, unsigned int* __restrict__ next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) break;
    int m = 0;
    while (m + 1 < nmem && mem[m + 1].item0 <= item) ++m;
    const EnsMember<T>& M = mem[m];
    const int local = item - M.item0;
    tiled_item<T, LIM, TT, TP>(M.sh, M.g, M.ph, M.Br, M.U, M.R, M.red, M.kchunk, local % M.ntiles,
                               local / M.ntiles, local, M.nitems, smem_raw);
    __syncthreads();  // shared memory and s_item are reused by the next item
  }
}

}  // namespace crn
