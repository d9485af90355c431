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
template <int NTHREADS>
__device__ void reduce_and_finalize(const double (&sum)[NV], double dtmin, const Reduce& red,
                                    double* scratch /* >= (NTHREADS/32) * RED_STRIDE doubles */) {
  constexpr int NW = NTHREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[NV + 1];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sum[q];
  v[NV] = dtmin;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    v[NV] = fmin(v[NV], __shfl_xor_sync(0xffffffffu, v[NV], off));
  }
  __syncthreads();  // scratch may alias buffers still in use
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q <= NV; ++q) scratch[warp * RED_STRIDE + q] = v[q];
  }
  __syncthreads();
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
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
    inner_ghost(wi, Br[col], (double)g.rhat[col], (double)g.rhat[cs + col],
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
    // ---- divide by the volume, gravity source [Sect. 2.2]
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
// production kernel: radial marching over a (theta, phi) tile
// ---------------------------------------------------------------------------
template <int TT, int TP>
struct TileDims {
  static constexpr int NT = TT * TP;           // threads = own columns
  static constexpr int HT = TT + 4, HP = TP + 4, HC = HT * HP;  // halo'd plane
  static constexpr int NFR = TT * TP;          // r faces per plane
  static constexpr int NFT = (TT + 1) * TP;    // theta faces per plane
  static constexpr int NFP = TT * (TP + 1);    // phi faces per plane
  static constexpr int NF = NV + 1;            // 9 fluxes + lambda |S|
  template <class T>
  static constexpr size_t smem_bytes() {
    return sizeof(T) * ((size_t)4 * NV * HC + (size_t)NF * (2 * NFR + NFT + NFP));
  }
};

template <class T, int LIM, int TT, int TP>
__global__ void __launch_bounds__(TT * TP)
residual_tiled(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br,
               const T* __restrict__ U, T* __restrict__ R, Reduce red, int kchunk) {
  using D = TileDims<TT, TP>;
  constexpr int NT = D::NT, HP = D::HP, HC = D::HC;
  constexpr int NFR = D::NFR, NFT = D::NFT, NFP = D::NFP, NF = D::NF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);   // [4][NV][HC]
  T* frb = ring + 4 * NV * HC;                // [2][NF][NFR]
  T* ftb = frb + 2 * NF * NFR;                // [NF][NFT]
  T* fpb = ftb + NF * NFT;                    // [NF][NFP]

  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t N = sh.ncell, cs = (int64_t)nt * np;
  const int tid = threadIdx.x;
  const int ntp = (np + TP - 1) / TP;
  const int j0 = (blockIdx.x / ntp) * TT, i0 = (blockIdx.x % ntp) * TP;
  const int k0 = blockIdx.y * kchunk;
  const int k1 = min(nr, k0 + kchunk);
  const int jj = tid / TP, ii = tid % TP;
  const int jo = j0 + jj, io = i0 + ii;
  const bool own = jo < nt && io < np;
  const int64_t ocol = own ? (int64_t)jo * np + io : 0;
  const int hown = (jj + 2) * HP + (ii + 2);

  auto slot = [&](int p) -> T* { return ring + ((p + 4) & 3) * (NV * HC); };

  // load plane p (0 <= p < nr) of the halo'd tile and recover its primitives
  auto load_plane = [&](int p) {
    T* dst = slot(p);
    const T* src = U + (int64_t)p * cs;
    for (int q = tid; q < HC; q += NT) {
      int j = j0 - 2 + q / HP, i = i0 - 2 + q % HP;
      map_column(j, i, nt, np);
      const int64_t c = (int64_t)j * np + i;
      T u[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = __ldg(src + v * N + c);
      recover(u, ph, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + q] = w[v];
    }
  };
  // ghost plane -1 (inner, low-E) or nr (outer) from the adjacent interior plane
  auto ghost_plane = [&](int p) {
    const T* srcp = slot(p < 0 ? 0 : nr - 1);
    T* dst = slot(p);
    for (int q = tid; q < HC; q += NT) {
      int j = j0 - 2 + q / HP, i = i0 - 2 + q % HP;
      map_column(j, i, nt, np);
      const int64_t c = (int64_t)j * np + i;
      T wi[NV], wg[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wi[v] = srcp[v * HC + q];
      if (p < 0)
        inner_ghost(wi, Br[c], (double)g.rhat[c], (double)g.rhat[cs + c], (double)g.rhat[2 * cs + c],
                    ph, wg);
      else
        outer_ghost(wi, g.rhat[c], g.rhat[cs + c], g.rhat[2 * cs + c], ph, wg);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + q] = wg[v];
    }
  };
  auto put_face = [&](T* buf, int stride, int q, const T (&f)[NV], T la) {
#pragma unroll
    for (int v = 0; v < NV; ++v) buf[v * stride + q] = f[v];
    buf[NV * stride + q] = la;
  };
  auto zero_face = [&](T* buf, int stride, int q) {
#pragma unroll
    for (int v = 0; v <= NV; ++v) buf[v * stride + q] = (T)0;
  };
  // r face between planes kf and kf + 1 for own column -> frb[(kf & 1)]
  auto r_face = [&](int kf) {
    T* buf = frb + (kf & 1) * (NF * NFR);
    if (!own) { zero_face(buf, NFR, tid); return; }
    T wl[NV], wr[NV];
    if (kf < 0 || kf >= nr - 1) {
      const T* a = slot(kf);
      const T* b = slot(kf + 1);
#pragma unroll
      for (int v = 0; v < NV; ++v) { wl[v] = a[v * HC + hown]; wr[v] = b[v * HC + hown]; }
    } else {
      T a[NV], b[NV], c[NV], d[NV];
      const T *pa = slot(kf - 1), *pb = slot(kf), *pc = slot(kf + 1), *pd = slot(kf + 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        a[v] = pa[v * HC + hown]; b[v] = pb[v * HC + hown];
        c[v] = pc[v * HC + hown]; d[v] = pd[v * HC + hown];
      }
      face_states<LIM>(a, b, c, d, g.inv_dm[kf], g.inv_dp[kf], g.hp[kf], g.inv_dm[kf + 1],
                       g.inv_dp[kf + 1], g.hm[kf + 1], ph.eps, wl, wr);
    }
    const T area = g.ra[kf + 1] * g.ar[jo];
    T f[NV], la;
    rusanov(wl, wr, g.nr[ocol], g.nr[cs + ocol], g.nr[2 * cs + ocol], area, ph, f, la);
    put_face(buf, NFR, tid, f, la);
  };

  // ---------------- preamble: planes k0-2 .. k0+1 and the r face k0 - 1/2
  for (int p = max(k0 - 2, 0); p <= min(k0 + 1, nr - 1); ++p) load_plane(p);
  __syncthreads();
  if (k0 - 2 <= -1) { ghost_plane(-1); }
  if (k0 + 1 >= nr) { ghost_plane(nr); }
  __syncthreads();
  r_face(k0 - 1);

  Acc<T> acc;
  acc.init();
  T dtm = (T)INFINITY;
  const T one = (T)1, half = (T)0.5;

  for (int k = k0; k < k1; ++k) {
    // ---- A: plane k + 2 enters the ring
    __syncthreads();
    if (k + 2 < nr) load_plane(k + 2);
    else if (k + 2 == nr) {
      // the outer ghost needs plane nr - 1, already in the ring
      ghost_plane(nr);
    }
    __syncthreads();
    // ---- C: every face of plane k, once
    for (int q = tid; q < NFR + NFT + NFP; q += NT) {
      if (q < NFR) {
        if (q == tid) r_face(k);  // q == tid for the r faces (NFR == NT)
      } else if (q < NFR + NFT) {
        const int qt = q - NFR;
        const int frow = qt / TP, col = qt % TP;
        const int jf = j0 + frow, ic = i0 + col;
        if (jf <= 0 || jf >= nt || ic >= np) { zero_face(ftb, NFT, qt); continue; }
        const T* pl = slot(k);
        T a[NV], b[NV], c[NV], d[NV], wl[NV], wr[NV];
        const int h0 = frow * HP + col + 2;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          a[v] = pl[v * HC + h0]; b[v] = pl[v * HC + h0 + HP];
          c[v] = pl[v * HC + h0 + 2 * HP]; d[v] = pl[v * HC + h0 + 3 * HP];
        }
        face_states<LIM>(a, b, c, d, one, one, half, one, one, half, ph.eps, wl, wr);
        const int64_t fc = (int64_t)jf * np + ic;
        const int64_t ts = (int64_t)(nt + 1) * np;
        const T area = g.rb[k] * g.at[jf];
        T f[NV], la;
        rusanov(wl, wr, g.nth[fc], g.nth[ts + fc], g.nth[2 * ts + fc], area, ph, f, la);
        put_face(ftb, NFT, qt, f, la);
      } else {
        const int qp = q - NFR - NFT;
        const int row = qp / (TP + 1), fcol = qp % (TP + 1);
        const int jr = j0 + row, ifc = i0 + fcol;
        if (jr >= nt || ifc > np) { zero_face(fpb, NFP, qp); continue; }
        const T* pl = slot(k);
        T a[NV], b[NV], c[NV], d[NV], wl[NV], wr[NV];
        const int h0 = (row + 2) * HP + fcol;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          a[v] = pl[v * HC + h0]; b[v] = pl[v * HC + h0 + 1];
          c[v] = pl[v * HC + h0 + 2]; d[v] = pl[v * HC + h0 + 3];
        }
        face_states<LIM>(a, b, c, d, one, one, half, one, one, half, ph.eps, wl, wr);
        const int iw = ifc == np ? 0 : ifc;
        const T area = g.rb[k] * g.dtheta;
        T f[NV], la;
        rusanov(wl, wr, g.nph[iw], g.nph[np + iw], (T)0, area, ph, f, la);
        put_face(fpb, NFP, qp, f, la);
      }
    }
    __syncthreads();
    // ---- E: gather the six faces of cell (k, jo, io)
    if (own) {
      const T* lo = frb + ((k - 1) & 1) * (NF * NFR);
      const T* hi = frb + (k & 1) * (NF * NFR);
      const int tl = jj * TP + ii, tu = tl + TP;
      const int pl = jj * (TP + 1) + ii, pu = pl + 1;
      T r[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        r[v] = (lo[v * NFR + tid] - hi[v * NFR + tid]) + (ftb[v * NFT + tl] - ftb[v * NFT + tu])
               + (fpb[v * NFP + pl] - fpb[v * NFP + pu]);
      const T lam = (lo[NV * NFR + tid] + hi[NV * NFR + tid]) + (ftb[NV * NFT + tl] + ftb[NV * NFT + tu])
                    + (fpb[NV * NFP + pl] + fpb[NV * NFP + pu]);
      const T vol = g.rv[k] * g.av[jo];
      const T ivol = one / vol;
#pragma unroll
      for (int v = 0; v < NV; ++v) r[v] *= ivol;
      const T* wc = slot(k);
      const T rho = wc[hown], vx = wc[HC + hown], vy = wc[2 * HC + hown], vz = wc[3 * HC + hown];
      const T gk = -g.grav[k];
      const T gx = gk * g.rhat[ocol], gy = gk * g.rhat[cs + ocol], gz = gk * g.rhat[2 * cs + ocol];
      r[1] += rho * gx;
      r[2] += rho * gy;
      r[3] += rho * gz;
      r[7] += rho * (vx * gx + vy * gy + vz * gz);
      const int64_t cell = (int64_t)k * cs + ocol;
      T chk = (T)0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R[v * N + cell] = r[v];
        acc.add(v, r[v]);
        chk += r[v] * r[v];
      }
      const T dtc = vol / lam;
      dtm = dtc < dtm ? dtc : dtm;
      const T pc = wc[7 * HC + hown];
      if (!(rho > (T)0) || !(pc > (T)0) || !(chk == chk) || chk > (T)1e300 * (T)1e300)
        flag_bad(red, cell);
    }
  }
  // ---------------- reductions
  double tot[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = acc.total(v);
  double* scratch = reinterpret_cast<double*>(smem_raw);
  reduce_and_finalize<NT>(tot, (double)dtm, red, scratch);
}

}  // namespace crn
