// nk.cu -- matrix-free Newton-Krylov pseudo-transient steady solver.
//
// The implicit pseudo-time iteration of Sect. 2.1 (backward Euler with local
// time steps, linearised once per step):
//
//   (diag(1 / dtau_c) - dR/dU) dU = R(U),    dtau_c = CFL dt_c,
//   dt_c = V_c / sum_f max(|V_c . n_f| + c_f(W_c, n_f), c_h) |S_f|,
//
// solved by restarted GMRES on the right-preconditioned operator
// y -> (D - J) P^-1 y (dU = P^-1 y) with P = diag(1/dtau) (P^-1 y = dtau . y) or
// P the radial line-implicit approximation of (D - J): per radial column a
// tridiagonal of the diagonal D + (1/V) sum_f lambda_f |S_f| / 2 and the
// couplings -lambda_r |S_r| / (2 V) to the radial neighbours, the Rusanov
// dissipation part of the Jacobian, solved by the Thomas algorithm (factored
// once per step, then one substitution per Krylov step); the
// Jacobian-vector product
// taken from residual evaluations of this library,
//   J z ~ (R(U + eps z) - R(U - eps z)) / (2 eps)   (or the forward difference),
// eps = min(b min_e (|u_e| + s_v(e)) / |z_e|, min_c p_c / (4 |dp_lin,c(z)|)),
// so that no entry of the state moves by more than the fraction b of its own
// size (s_v = 1e-3 x (the mean |u| of its variable + the mean |u| over all
// nine variables)) and no cell's pressure by more than a quarter.  The step is
// then limited to a relative change of rho and of the linearised p of at most
// omega per cell, and halved while any cell of U + alpha dU would keep less
// than a tenth of its density or pressure.  The CFL law of Sect. 4.1
// (start at 2, double every few steps, up to 128) drives crn_steady_solve.
//
// Every vector operation is a kernel of this file, in FP64 except the
// Gram-Schmidt dots and updates of an FP32 Krylov basis (basis_fp32);
// reductions go through per-block partials summed in a fixed order, so a
// solve is bitwise reproducible.  The host runs the GMRES recurrences (Hessenberg, Givens) and
// synchronises the stream once or twice per Krylov step to read the dots.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "corona_internal.h"
#include "fp_bits.cuh"

namespace crn {

namespace {

constexpr int NKB = 256;  // threads per block of the vector kernels
// a Newton step keeps at least this fraction of every cell's density and pressure
constexpr double kKeepFrac = 0.1;
constexpr int MD = 8;     // vectors per multi-dot launch

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// block sum of K values per thread into part[(row + k) * nblk + blockIdx.x]
template <int K>
__device__ __forceinline__ void block_sum_rows(double (&a)[K], double* part, int nblk, int row,
                                               int cnt) {
  __shared__ double sm[(NKB / 32) * K];
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sm[wid * K + k] = a[k];
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int q = 0; q < NKB / 32; ++q) s += sm[q * K + threadIdx.x];
    part[(size_t)(row + threadIdx.x) * nblk + blockIdx.x] = s;
  }
}

// partial dots <V_(i0+t), w>, t < cnt, into rows row_v + t; with ww also
// <w, w> into row row_ww
__global__ void __launch_bounds__(NKB)
mdot_kernel(const double* __restrict__ V, int64_t n, int i0, int cnt, const double* __restrict__ w,
            double* __restrict__ part, int nblk, int row_v, int ww, int row_ww) {
  double a[MD + 1];
#pragma unroll
  for (int t = 0; t <= MD; ++t) a[t] = 0.0;
  const int64_t stride = (int64_t)nblk * NKB;
  // two elements per trip: their loads are in flight together, so that the
  // FMAs (bound by the FP64 pipe) overlap the memory latency
#pragma unroll 2
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) {
    const double we = w[e];
#pragma unroll
    for (int t = 0; t < MD; ++t)
      if (t < cnt) a[t] += V[(int64_t)(i0 + t) * n + e] * we;
    a[MD] += we * we;
  }
  double b[MD];
#pragma unroll
  for (int t = 0; t < MD; ++t) b[t] = a[t];
  block_sum_rows<MD>(b, part, nblk, row_v, cnt);
  if (ww) {
    double c[1] = {a[MD]};
    __syncthreads();
    block_sum_rows<1>(c, part, nblk, row_ww, 1);
  }
}

// out[row] = sum over blocks of part[row][.] (sum, max or min), one block per row
__global__ void __launch_bounds__(NKB)
finish_kernel(const double* __restrict__ part, int nblk, int row0, double* __restrict__ out, int op) {
  __shared__ double sm[NKB];
  const int row = row0 + blockIdx.x;
  double s = op == 0 ? 0.0 : (op == 1 ? -INFINITY : INFINITY);
  for (int q = threadIdx.x; q < nblk; q += NKB) {
    const double v = part[(size_t)row * nblk + q];
    s = op == 0 ? s + v : (op == 1 ? fmax(s, v) : fmin(s, v));
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int h = NKB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const double o = sm[threadIdx.x + h];
      sm[threadIdx.x] = op == 0 ? sm[threadIdx.x] + o : (op == 1 ? fmax(sm[threadIdx.x], o) : fmin(sm[threadIdx.x], o));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[row] = sm[0];
}

// w += sum_t coef[t] V_t (V FP64, or the FP32 basis into an FP64 w)
template <class TV>
__global__ void __launch_bounds__(NKB)
maxpy_kernel(double* __restrict__ w, const TV* __restrict__ V, int64_t n,
             const double* __restrict__ coef, int cnt) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) {
    double s = w[e];
    for (int t = 0; t < cnt; ++t) s += coef[t] * (double)V[(int64_t)t * n + e];
    w[e] = s;
  }
}

// ---- FP32 Krylov basis: the orthogonalisation on the FP32 pipe (GB300 runs
// FP64 FMAs at 1/64 of the FP32 rate, which bounds the FP64 multi-dot and
// update); sums over a thread's elements in FP32, across threads in FP64

// partial dots <Vf_(i0+t), wf>, t < cnt, into rows row_v + t; with ww <wf, wf>
__global__ void __launch_bounds__(NKB)
mdot32_kernel(const float* __restrict__ V, int64_t n, int i0, int cnt, const float* __restrict__ w,
              double* __restrict__ part, int nblk, int row_v, int ww, int row_ww) {
  float a[MD + 1];
#pragma unroll
  for (int t = 0; t <= MD; ++t) a[t] = 0.f;
  const int64_t stride = (int64_t)nblk * NKB;
#pragma unroll 2
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) {
    const float we = w[e];
#pragma unroll
    for (int t = 0; t < MD; ++t)
      if (t < cnt) a[t] = fmaf(V[(int64_t)(i0 + t) * n + e], we, a[t]);
    a[MD] = fmaf(we, we, a[MD]);
  }
  double b[MD];
#pragma unroll
  for (int t = 0; t < MD; ++t) b[t] = (double)a[t];
  block_sum_rows<MD>(b, part, nblk, row_v, cnt);
  if (ww) {
    double c[1] = {(double)a[MD]};
    __syncthreads();
    block_sum_rows<1>(c, part, nblk, row_ww, 1);
  }
}

// wf += sum_t coef[t] Vf_t in FP32
__global__ void __launch_bounds__(NKB)
maxpy32_kernel(float* __restrict__ w, const float* __restrict__ V, int64_t n,
               const float* __restrict__ coef, int cnt) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) {
    float s = w[e];
    for (int t = 0; t < cnt; ++t) s = fmaf(coef[t], V[(int64_t)t * n + e], s);
    w[e] = s;
  }
}

// y = (float)(a x); x FP64 (a new Arnoldi vector, a restart vector) or FP32
template <class TX>
__global__ void __launch_bounds__(NKB)
to32_kernel(float* y, const TX* x, double a, int64_t n) {  // y may alias x when TX = float
  const int64_t stride = (int64_t)gridDim.x * NKB;
  if (sizeof(TX) == 4) {
    const float af = (float)a;
    for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) y[e] = af * (float)x[e];
  } else {
    for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) y[e] = (float)(a * (double)x[e]);
  }
}

__global__ void __launch_bounds__(NKB)
scale_kernel(double* y, const double* x, double a, int64_t n) {  // y may alias x
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) y[e] = a * x[e];
}

// y = b - x (y may alias x)
__global__ void __launch_bounds__(NKB)
sub_kernel(double* y, const double* b, const double* x, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) y[e] = b[e] - x[e];
}

// y += x
__global__ void __launch_bounds__(NKB)
add_kernel(double* y, const double* x, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) y[e] += x[e];
}

// w = z / dtau - w: the shifted adjoint operator (D - J^T) z from w = J^T z
// (D = diag(1 / dtau), one dtau per cell shared by its nine variables)
__global__ void __launch_bounds__(NKB)
shift_combine_kernel(double* __restrict__ w, const double* __restrict__ z, const double* __restrict__ dtau,
                     int64_t N, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) w[e] = z[e] / dtau[e % N] - w[e];
}

// per-variable partial sums of |u| (rows 0..8)
__global__ void __launch_bounds__(NKB)
absmean_kernel(const double* __restrict__ U, int64_t N, double* __restrict__ part, int nblk, int row) {
  double a[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) a[v] = 0.0;
  const int64_t stride = (int64_t)nblk * NKB;
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
#pragma unroll
    for (int v = 0; v < NV; ++v) a[v] += fabs(U[v * N + c]);
  }
  block_sum_rows<NV>(a, part, nblk, row, NV);
}

// reciprocal good to about 20 bits (PTX rcp.approx.ftz.f64), for the ratios
// that only set the finite-difference step: an IEEE division costs several
// slots of the slow FP64 pipe, and the step needs its magnitude only
__device__ __forceinline__ double rcp_coarse(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

// z = dtau . v (dtau per cell, shared by its nine variables).  With want_min,
// two partial minima for the finite-difference step: over entries of
// (|u| + s_v) / |z| into row `row`, and over cells of p / |dp_lin(z)| into
// row `row` + 1 (dp_lin the linearised pressure change along z)
template <class TV>
__global__ void __launch_bounds__(NKB)
precond_kernel(const TV* __restrict__ v, const double* __restrict__ dtau, int64_t N,
               double* __restrict__ z, const double* __restrict__ U, const double* __restrict__ sumabs,
               double gm1, double* __restrict__ part, int nblk, int row, int want_min) {
  double m = INFINITY, mp = INFINITY;
  const int64_t stride = (int64_t)nblk * NKB;
  // floors s_v = 1e-3 (mean |u_v| + mean |u| over the nine variables): never
  // zero, also for a variable that vanishes everywhere (psi of a start state)
  double s[NV];
  if (want_min) {
    double tot = 0.0;
#pragma unroll
    for (int q = 0; q < NV; ++q) tot += sumabs[q];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = 1e-3 * (sumabs[q] + tot / NV) / (double)N;
  }
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
    // dtau null: v already is the direction z (statistics only)
    const double d = dtau ? dtau[c] : 1.0;
    double zz[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      zz[q] = d * (double)v[q * N + c];
      if (dtau) z[q * N + c] = zz[q];
    }
    if (!want_min) continue;
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      u[q] = U[q * N + c];
      if (zz[q] != 0.0) m = fmin(m, (fabs(u[q]) + s[q]) * rcp_coarse(fabs(zz[q])));
    }
    const double ir = rcp_coarse(u[0]);
    const double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
    const double p = gm1 * (u[7] - 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz) -
                            0.5 * (u[4] * u[4] + u[5] * u[5] + u[6] * u[6]));
    const double dp = gm1 * (zz[7] - (vx * zz[1] + vy * zz[2] + vz * zz[3]) +
                             0.5 * (vx * vx + vy * vy + vz * vz) * zz[0] -
                             (u[4] * zz[4] + u[5] * zz[5] + u[6] * zz[6]));
    if (dp != 0.0) mp = fmin(mp, p * rcp_coarse(fabs(dp)));
    // second order: p(U + e z) = p + e dp - e^2 gm1 Q + ..., Q = |z_B|^2 / 2 +
    // |z_m - V z_rho|^2 / (2 rho); with e <= mp / 4 this keeps e^2 gm1 Q <= p / 4
    const double wx = zz[1] - vx * zz[0], wy = zz[2] - vy * zz[0], wz = zz[3] - vz * zz[0];
    const double Q = 0.5 * (zz[4] * zz[4] + zz[5] * zz[5] + zz[6] * zz[6]) +
                     0.5 * (wx * wx + wy * wy + wz * wz) * ir;
    if (Q > 0.0 && p > 0.0) mp = fmin(mp, 2.0 * sqrt(p * rcp_coarse(gm1 * Q)));
  }
  if (!want_min) return;
  __shared__ double sm[2][NKB];
  sm[0][threadIdx.x] = m;
  sm[1][threadIdx.x] = mp;
  __syncthreads();
  for (int h = NKB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sm[0][threadIdx.x] = fmin(sm[0][threadIdx.x], sm[0][threadIdx.x + h]);
      sm[1][threadIdx.x] = fmin(sm[1][threadIdx.x], sm[1][threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[(size_t)row * nblk + blockIdx.x] = sm[0][0];
    part[(size_t)(row + 1) * nblk + blockIdx.x] = sm[1][0];
  }
}

// eps = min(b * entry ratio, p ratio / 4) (1 if z = 0), written to out[dst]
__global__ void eps_kernel(double* out, int src, int dst, double b) {
  const double m = b * out[src];
  const double mp = 0.25 * out[src + 1];
  const double e = fmin(m, mp);
  out[dst] = isfinite(e) && e > 0.0 ? e : (isfinite(m) ? m : 1.0);
}

// ut = (T)(U + sign eps z) (eps = 0 without z)
template <class T>
__global__ void __launch_bounds__(NKB)
perturb_kernel(const double* __restrict__ U, const double* __restrict__ z,
               const double* __restrict__ eps, double sign, int64_t n, T* __restrict__ ut) {
  const double ee = z ? sign * *eps : 0.0;
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride)
    ut[e] = (T)(z ? U[e] + ee * z[e] : U[e]);
}

// w = v - (R(U + eps z) - R(U)) / eps (forward difference, div = 1) or
// w = v - (R(U + eps z) - R(U - eps z)) / (2 eps) (central difference, div = 2)
template <class T, class TV = double>
__global__ void __launch_bounds__(NKB)
jvp_combine_kernel(const TV* __restrict__ v, const T* __restrict__ rp, const T* __restrict__ rb,
                   const double* __restrict__ eps, double div, int64_t n, double* __restrict__ w,
                   const double* __restrict__ dinv = nullptr, const double* __restrict__ z = nullptr,
                   int64_t N = 1) {
  const double ie = 1.0 / (div * *eps);
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) {
    // with dinv: the D z term of (D - J) z for a general right preconditioner
    const double first = dinv ? dinv[e % N] * z[e] : (v ? (double)v[e] : 0.0);
    w[e] = first - ((double)rp[e] - (double)rb[e]) * ie;
  }
}

__global__ void __launch_bounds__(NKB)
widen_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) y[e] = (double)x[e];
}

__device__ __forceinline__ void prim_of(const double* __restrict__ U, int64_t N, int64_t c, double gm1,
                                        double& rho, double (&v)[3], double (&b)[3], double& p) {
  rho = U[c];
  const double ir = 1.0 / rho;
  v[0] = U[N + c] * ir; v[1] = U[2 * N + c] * ir; v[2] = U[3 * N + c] * ir;
  b[0] = U[4 * N + c]; b[1] = U[5 * N + c]; b[2] = U[6 * N + c];
  p = gm1 * (U[7 * N + c] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) -
             0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]));
}

// partial max over cells of max(|d rho| / rho, |dp_lin| / p),
// dp_lin = (gamma - 1)(dE - V.dm + |V|^2 drho / 2 - B.dB)
__global__ void __launch_bounds__(NKB)
relchange_kernel(const double* __restrict__ U, const double* __restrict__ dU, int64_t N, double gm1,
                 double* __restrict__ part, int nblk, int row) {
  double m = 0.0;
  const int64_t stride = (int64_t)nblk * NKB;
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
    double rho, v[3], b[3], p;
    prim_of(U, N, c, gm1, rho, v, b, p);
    const double drho = dU[c];
    const double dp = gm1 * (dU[7 * N + c] - (v[0] * dU[N + c] + v[1] * dU[2 * N + c] + v[2] * dU[3 * N + c]) +
                             0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * drho -
                             (b[0] * dU[4 * N + c] + b[1] * dU[5 * N + c] + b[2] * dU[6 * N + c]));
    const double r = fmax(fabs(drho) / rho, fabs(dp) / p);
    m = isnan(r) ? INFINITY : fmax(m, r);
  }
  __shared__ double sm[NKB];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int h = NKB / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)row * nblk + blockIdx.x] = sm[0];
}

// partial count of cells of U + alpha dU with rho <= 0, p <= 0 or not finite
__global__ void __launch_bounds__(NKB)
badcount_kernel(const double* __restrict__ U, const double* __restrict__ dU, double alpha, int64_t N,
                double gm1, double* __restrict__ part, int nblk, int row) {
  double cnt[1] = {0.0};
  const int64_t stride = (int64_t)nblk * NKB;
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = U[q * N + c] + alpha * dU[q * N + c];
    const double rho = u[0];
    const double ir = 1.0 / rho;
    const double p = gm1 * (u[7] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * ir -
                            0.5 * (u[4] * u[4] + u[5] * u[5] + u[6] * u[6]));
    // the old state's density and pressure: a step may not take away more
    // than (1 - kKeepFrac) of either in any cell
    double r0, v0[3], b0[3], p0;
    prim_of(U, N, c, gm1, r0, v0, b0, p0);
    if (!(rho > kKeepFrac * r0) || !(p > kKeepFrac * p0) || !isfinite(p)) cnt[0] += 1.0;
  }
  block_sum_rows<1>(cnt, part, nblk, row, 1);
}

// U += alpha dU
__global__ void __launch_bounds__(NKB)
apply_kernel(double* __restrict__ U, const double* __restrict__ dU, double alpha, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) U[e] += alpha * dU[e];
}

// dtau_c = cfl V_c / sum_f max(|V.n_f| + c_f, c_h) |S_f| from the cell's own
// FP64 state, the grid's face-area factors and unit normals
template <class T>
__global__ void __launch_bounds__(NKB)
local_dt_kernel(Shape sh, Geo<T> g, double gamma, double ch, const double* __restrict__ U, double cfl,
                double* __restrict__ dtau) {
  const int64_t N = sh.ncell;
  const int64_t cs = (int64_t)sh.nt * sh.np;
  const int64_t ts = (int64_t)(sh.nt + 1) * sh.np;
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
    const int i = (int)(c % sh.np);
    const int j = (int)((c / sh.np) % sh.nt);
    const int k = (int)(c / cs);
    const int64_t col = (int64_t)j * sh.np + i;
    double rho, v[3], b[3], p;
    prim_of(U, N, c, gamma - 1.0, rho, v, b, p);
    const double ir = 1.0 / rho;
    const double a2 = gamma * p * ir;
    const double b2 = (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]) * ir;
    auto lam = [&](double nx, double ny, double nz) {
      const double un = v[0] * nx + v[1] * ny + v[2] * nz;
      const double bn = b[0] * nx + b[1] * ny + b[2] * nz;
      const double s = a2 + b2;
      const double disc = fmax(s * s - 4.0 * a2 * bn * bn * ir, 0.0);
      return fmax(fabs(un) + sqrt(0.5 * (s + sqrt(disc))), ch);
    };
    double sum = 0.0;
    {  // r faces k and k + 1 share the column's unit normal
      const double l = lam((double)g.nr[col], (double)g.nr[cs + col], (double)g.nr[2 * cs + col]);
      sum += l * ((double)g.ra[k] + (double)g.ra[k + 1]) * (double)g.ar[j];
    }
    for (int jf = j; jf <= j + 1; ++jf) {
      const double area = (double)g.rb[k] * (double)g.at[jf];
      if (area == 0.0) continue;  // pole faces
      const int64_t fc = (int64_t)jf * sh.np + i;
      sum += lam((double)g.nth[fc], (double)g.nth[ts + fc], (double)g.nth[2 * ts + fc]) * area;
    }
    for (int ifc = i; ifc <= i + 1; ++ifc) {
      const int iw = ifc % sh.np;
      sum += lam((double)g.nph[iw], (double)g.nph[sh.np + iw], 0.0) * (double)g.rb[k] * (double)g.dtheta;
    }
    dtau[c] = cfl * ((double)g.rv[k] * (double)g.av[j]) / sum;
  }
}

// coefficients of the radial line preconditioner P ~ (D - J): per cell the
// D entry dinv = 1/dtau, the diagonal dinv + (1/V) sum_f lambda_f |S_f| / 2 and
// the couplings -lambda_r |S_r| / (2 V) to the radial neighbours (the Rusanov
// dissipation part of dR/dU), lambda from the cell's own state as for dt_c
template <class T>
__global__ void __launch_bounds__(NKB)
line_coef_kernel(Shape sh, Geo<T> g, double gamma, double ch, const double* __restrict__ U, double cfl,
                 double* __restrict__ dinv, double* __restrict__ di, double* __restrict__ lo,
                 double* __restrict__ up) {
  const int64_t N = sh.ncell;
  const int64_t cs = (int64_t)sh.nt * sh.np;
  const int64_t ts = (int64_t)(sh.nt + 1) * sh.np;
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
    const int i = (int)(c % sh.np);
    const int j = (int)((c / sh.np) % sh.nt);
    const int k = (int)(c / cs);
    const int64_t col = (int64_t)j * sh.np + i;
    double rho, v[3], b[3], p;
    prim_of(U, N, c, gamma - 1.0, rho, v, b, p);
    const double ir = 1.0 / rho;
    const double a2 = gamma * p * ir;
    const double b2 = (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]) * ir;
    auto lam = [&](double nx, double ny, double nz) {
      const double un = v[0] * nx + v[1] * ny + v[2] * nz;
      const double bn = b[0] * nx + b[1] * ny + b[2] * nz;
      const double s = a2 + b2;
      const double disc = fmax(s * s - 4.0 * a2 * bn * bn * ir, 0.0);
      return fmax(fabs(un) + sqrt(0.5 * (s + sqrt(disc))), ch);
    };
    const double lr = lam((double)g.nr[col], (double)g.nr[cs + col], (double)g.nr[2 * cs + col]);
    const double slo = lr * (double)g.ra[k] * (double)g.ar[j];
    const double sup = lr * (double)g.ra[k + 1] * (double)g.ar[j];
    double sum = slo + sup;
    for (int jf = j; jf <= j + 1; ++jf) {
      const double area = (double)g.rb[k] * (double)g.at[jf];
      if (area == 0.0) continue;
      const int64_t fc = (int64_t)jf * sh.np + i;
      sum += lam((double)g.nth[fc], (double)g.nth[ts + fc], (double)g.nth[2 * ts + fc]) * area;
    }
    for (int ifc = i; ifc <= i + 1; ++ifc) {
      const int iw = ifc % sh.np;
      sum += lam((double)g.nph[iw], (double)g.nph[sh.np + iw], 0.0) * (double)g.rb[k] * (double)g.dtheta;
    }
    const double iv = 1.0 / ((double)g.rv[k] * (double)g.av[j]);
    dinv[c] = sum * iv / cfl;
    di[c] = dinv[c] + 0.5 * sum * iv;
    lo[c] = k > 0 ? -0.5 * slo * iv : 0.0;
    up[c] = k < sh.nr - 1 ? -0.5 * sup * iv : 0.0;
  }
}

// z = P^-1 v along every radial column (Thomas algorithm, the nine variables
// share the tridiagonal); one thread per column; cp: N doubles of scratch
// the adjoint's preconditioner P_a = -(L)^T ~ J^T from the forward line
// coefficients taken at infinite CFL (L = diag, lower, upper in slots 1, 2, 3):
// lower_T(k) = -upper(k - 1) -> slot 0, upper_T(k) = -lower(k + 1) -> slot 5,
// diag_T = -diag in place
__global__ void __launch_bounds__(NKB)
line_transpose_kernel(Shape sh, double* __restrict__ L) {
  const int64_t N = sh.ncell, cs = (int64_t)sh.nt * sh.np;
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t c = (int64_t)blockIdx.x * NKB + threadIdx.x; c < N; c += stride) {
    const int k = (int)(c / cs);
    L[c] = k > 0 ? -L[3 * N + c - cs] : 0.0;
    L[5 * N + c] = k < sh.nr - 1 ? -L[2 * N + c + cs] : 0.0;
  }
}

__global__ void __launch_bounds__(NKB)
negate_kernel(double* __restrict__ x, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * NKB;
  for (int64_t e = (int64_t)blockIdx.x * NKB + threadIdx.x; e < n; e += stride) x[e] = -x[e];
}

// Thomas factorisation of every radial line, once per set of coefficients:
// m_0 = d_0, m_k = d_k - l_k c_(k-1) with c_k = u_k / m_k; stores c_k and
// 1/m_k.  One thread per column (the recurrence runs along r).
__global__ void __launch_bounds__(NKB)
line_factor_kernel(Shape sh, const double* __restrict__ lo, const double* __restrict__ di,
                   const double* __restrict__ up, double* __restrict__ cp, double* __restrict__ im) {
  const int64_t cs = (int64_t)sh.nt * sh.np;
  const int64_t col = (int64_t)blockIdx.x * NKB + threadIdx.x;
  if (col >= cs) return;
  double c = 0.0;
  for (int k = 0; k < sh.nr; ++k) {
    const int64_t q = (int64_t)k * cs + col;
    const double inv = 1.0 / (k == 0 ? di[q] : di[q] - lo[q] * c);
    c = up[q] * inv;
    cp[q] = c;
    im[q] = inv;
  }
}

// z = P^-1 v along every radial column from the factors: forward
// y_k = (v_k - l_k y_(k-1)) / m_k, backward z_k = y_k - c_k z_(k+1).  One
// thread per (variable, column): the nine right-hand sides share the factors,
// and 9 n_theta n_phi threads keep every SM busy; the loads along r do not
// depend on the recurrence and are issued ahead of it.
// an FP32 Krylov vector widens on the integer pipe (exact): the FP64 pipe,
// which also runs the conversion instruction, carries the recurrence
__device__ __forceinline__ double as_double(float x) { return widen_f32(x); }
__device__ __forceinline__ double as_double(double x) { return x; }

template <class TV>
__global__ void __launch_bounds__(NKB)
line_solve_kernel(Shape sh, const double* __restrict__ lo, const double* __restrict__ cp,
                  const double* __restrict__ im, const TV* __restrict__ v, double* __restrict__ z) {
  const int64_t cs = (int64_t)sh.nt * sh.np, N = sh.ncell;
  const int64_t t = (int64_t)blockIdx.x * NKB + threadIdx.x;
  if (t >= NV * cs) return;
  const int64_t q = t / cs, col = t - q * cs;
  const TV* __restrict__ vq = v + q * N;
  double* __restrict__ zq = z + q * N;
  double y = as_double(vq[col]) * im[col];
  zq[col] = y;
#pragma unroll 4
  for (int k = 1; k < sh.nr; ++k) {
    const int64_t c = (int64_t)k * cs + col;
    y = fma(-lo[c], y, as_double(vq[c])) * im[c];
    zq[c] = y;
  }
#pragma unroll 4
  for (int k = sh.nr - 2; k >= 0; --k) {
    const int64_t c = (int64_t)k * cs + col;
    y = fma(-cp[c], y, zq[c]);
    zq[c] = y;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct NkWork {
  int m = 0;          // Krylov dimension the basis holds
  int64_t n = 0;      // 9 N
  int nblk = 0;       // blocks of the reduction kernels (fixed: deterministic sums)
  int rows = 0;       // rows of the partials / out arrays
  double* V = nullptr;     // (m + 1) x n basis
  double* z = nullptr;     // n: preconditioned direction, then dU
  double* x = nullptr;     // n: GMRES solution y
  double* b = nullptr;     // n: R(U) in FP64
  double* w = nullptr;     // n: Arnoldi vector
  void* ut = nullptr;      // n of T: cast / perturbed state
  void* rt = nullptr;      // n of T: perturbed residual
  void* rb = nullptr;      // n of T: base residual (FP32 grids) / R(U - eps z) (FP64 grids)
  void* rm = nullptr;      // n of T: R(U - eps z) (FP32 grids)
  double* dtau = nullptr;  // N
  double* line = nullptr;  // 7N: radial line preconditioner (dinv, diag, lower, upper, the
                           //     factors c_k, upper of the transposed lines for the adjoint,
                           //     the inverse pivots 1/m_k)
  float* Vf = nullptr;     // (m + 1) n: the FP32 Krylov basis (allocated on first use)
  float* wf = nullptr;     // n: the FP32 Arnoldi vector
  float* coef32 = nullptr; // m + 2 FP32 coefficients
  double* part = nullptr;  // rows x nblk partials
  double* out = nullptr;   // rows reduced values
  double* coef = nullptr;  // m + 2 coefficients
  double* host = nullptr;  // pinned mirror of out
  double* adj = nullptr;   // 2n: the pseudo-time adjoint's lambda and residual (first use)
  double* fv = nullptr;    // (mf + 1) n: outer FGMRES basis of the pseudo-time adjoint
  double* fz = nullptr;    // mf n: its preconditioned directions
  int mf = 0;
};

void nk_free(NkWork* w) {
  if (!w) return;
  cudaFree(w->V); cudaFree(w->z); cudaFree(w->x); cudaFree(w->b); cudaFree(w->w);
  cudaFree(w->ut); cudaFree(w->rt); cudaFree(w->rb); cudaFree(w->rm); cudaFree(w->dtau);
  cudaFree(w->line);
  cudaFree(w->Vf); cudaFree(w->wf); cudaFree(w->coef32);
  cudaFree(w->part); cudaFree(w->out); cudaFree(w->coef);
  cudaFree(w->adj);
  cudaFree(w->fv); cudaFree(w->fz);
  cudaFreeHost(w->host);
  delete w;
}

namespace {

// rows of the out array beyond the m + 2 dot rows
struct Rows {
  int ww, sumabs, minr, eps, relmax, bad, total;
  explicit Rows(int m) {
    ww = m + 1;
    sumabs = m + 2;
    minr = sumabs + NV;  // two rows: entry ratio, pressure ratio
    eps = minr + 2;
    relmax = eps + 1;
    bad = relmax + 1;
    total = bad + 1;
  }
};

int report(int code, const std::string& msg) { return report_error(code, msg.c_str()); }

// the FP32 Krylov basis of a workspace (allocated on first use)
cudaError_t ensure_basis32(NkWork* w) {
  if (w->Vf) return cudaSuccess;
  cudaError_t e = cudaMalloc(&w->Vf, sizeof(float) * (size_t)(w->m + 1) * w->n);
  if (e == cudaSuccess) e = cudaMalloc(&w->wf, sizeof(float) * w->n);
  if (e == cudaSuccess) e = cudaMalloc(&w->coef32, sizeof(float) * (w->m + 2));
  if (e != cudaSuccess) {
    cudaFree(w->Vf); cudaFree(w->wf); cudaFree(w->coef32);
    w->Vf = nullptr; w->wf = nullptr; w->coef32 = nullptr;
  }
  return e;
}

bool use_basis32(const crn_nk_options& o) {
  return o.basis_fp32 == 1 || (o.basis_fp32 == -1 && o.lin_rtol >= 1e-4);
}

cudaError_t ensure_work(crn_grid* g, int m) {
  NkWork* w = g->nk;
  const int64_t N = g->shape.ncell, n = 9 * N;
  if (w && w->m >= m) return cudaSuccess;
  if (w) { nk_free(w); g->nk = nullptr; }
  w = new NkWork();
  g->nk = w;
  w->m = m;
  w->n = n;
  w->nblk = 4 * g->cfg.num_sms;
  w->rows = Rows(m).total;
  const size_t es = g->d.precision == CRN_FP64 ? 8 : 4;
  cudaError_t e = cudaMalloc(&w->V, sizeof(double) * (size_t)(m + 1) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->z, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->x, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->b, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->w, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->ut, es * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->rt, es * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->rb, es * n);
  if (e == cudaSuccess && es == 4) e = cudaMalloc(&w->rm, es * n);
  if (e == cudaSuccess) e = cudaMalloc(&w->dtau, sizeof(double) * N);
  if (e == cudaSuccess) e = cudaMalloc(&w->line, sizeof(double) * 7 * N);
  if (e == cudaSuccess) e = cudaMalloc(&w->part, sizeof(double) * (size_t)w->rows * w->nblk);
  if (e == cudaSuccess) e = cudaMalloc(&w->out, sizeof(double) * w->rows);
  if (e == cudaSuccess) e = cudaMalloc(&w->coef, sizeof(double) * (m + 2));
  if (e == cudaSuccess) e = cudaMallocHost(&w->host, sizeof(double) * w->rows);
  if (e != cudaSuccess) { nk_free(w); g->nk = nullptr; }
  return e;
}

// the solver context of one call
struct Ctx {
  crn_grid* g;
  NkWork* w;
  cudaStream_t st;
  Rows rows;
  int64_t N, n;
  unsigned grid;    // blocks of the elementwise kernels
  int launches = 0;
  int evals = 0;
  cudaError_t err = cudaSuccess;
  Ctx(crn_grid* gg, cudaStream_t s) : g(gg), w(gg->nk), st(s), rows(gg->nk->m), N(gg->shape.ncell),
                                      n(9 * gg->shape.ncell) {
    grid = (unsigned)std::min<int64_t>((n + NKB - 1) / NKB, (int64_t)g->cfg.num_sms * 16);
  }
  bool ok() { if (err == cudaSuccess) err = cudaGetLastError(); return err == cudaSuccess; }

  void finish(int row0, int nrows, int op) {
    finish_kernel<<<nrows, NKB, 0, st>>>(w->part, w->nblk, row0, w->out, op);
    ++launches;
  }
  // copy out[row0 .. row0 + cnt) to the host and wait
  void fetch(int row0, int cnt) {
    if (!ok()) return;
    err = cudaMemcpyAsync(w->host + row0, w->out + row0, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  }
  // h[t] = <V_t, v> for t < cnt (into out rows 0..cnt-1); with ww also <v, v>
  void dots(int cnt, const double* v, bool ww) { dots_on(w->V, cnt, v, ww); }
  void dots_on(const double* base, int cnt, const double* v, bool ww) {
    for (int i0 = 0; i0 < cnt || (i0 == 0 && ww); i0 += MD) {
      const int c = std::min(MD, cnt - i0);
      mdot_kernel<<<w->nblk, NKB, 0, st>>>(base, n, i0, std::max(c, 0), v, w->part, w->nblk, i0,
                                           (ww && i0 == 0) ? 1 : 0, rows.ww);
      ++launches;
      if (i0 + MD >= cnt) break;
    }
    if (cnt > 0) finish(0, cnt, 0);
    if (ww) finish(rows.ww, 1, 0);
  }
  double norm(const double* v) {
    dots(0, v, true);
    fetch(rows.ww, 1);
    return std::sqrt(std::max(w->host[rows.ww], 0.0));
  }
  // y += sum_t c[t] V_t
  void combine(double* y, const double* c, int cnt) { combine_on(y, w->V, c, cnt); }
  void combine_on(double* y, const double* base, const double* c, int cnt) {
    if (!ok() || cnt <= 0) return;
    // a copy from pageable memory returns once the source has been staged, so
    // c may be reused at once; stream order keeps coef intact for maxpy
    err = cudaMemcpyAsync(w->coef, c, sizeof(double) * cnt, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return;
    maxpy_kernel<double><<<grid, NKB, 0, st>>>(y, base, n, w->coef, cnt);
    ++launches;
  }
  // FP32 basis: h[t] = <Vf_t, vf> (rows 0..cnt-1), with ww also <vf, vf>
  void dots32(int cnt, const float* v, bool ww) {
    for (int i0 = 0; i0 < cnt || (i0 == 0 && ww); i0 += MD) {
      const int c = std::min(MD, cnt - i0);
      mdot32_kernel<<<w->nblk, NKB, 0, st>>>(w->Vf, n, i0, std::max(c, 0), v, w->part, w->nblk, i0,
                                             (ww && i0 == 0) ? 1 : 0, rows.ww);
      ++launches;
      if (i0 + MD >= cnt) break;
    }
    if (cnt > 0) finish(0, cnt, 0);
    if (ww) finish(rows.ww, 1, 0);
  }
  double norm32(const float* v) {
    dots32(0, v, true);
    fetch(rows.ww, 1);
    return std::sqrt(std::max(w->host[rows.ww], 0.0));
  }
  // vf += sum_t c[t] Vf_t in FP32
  void combine32(float* y, const double* c, int cnt) {
    if (!ok() || cnt <= 0) return;
    std::vector<float> cf(c, c + cnt);
    // from pageable memory the copy returns once cf has been staged
    err = cudaMemcpyAsync(w->coef32, cf.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return;
    maxpy32_kernel<<<grid, NKB, 0, st>>>(y, w->Vf, n, w->coef32, cnt);
    ++launches;
  }
  // x += sum_t c[t] Vf_t in FP64 (the solution update of a cycle)
  void combine_x32(double* y, const double* c, int cnt) {
    if (!ok() || cnt <= 0) return;
    err = cudaMemcpyAsync(w->coef, c, sizeof(double) * cnt, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return;
    maxpy_kernel<float><<<grid, NKB, 0, st>>>(y, w->Vf, n, w->coef, cnt);
    ++launches;
  }
  template <class TX>
  void to32(float* y, const TX* x, double a) {
    to32_kernel<TX><<<grid, NKB, 0, st>>>(y, x, a, n);
    ++launches;
  }
  void residual(const void* u, void* r) {
    int nl = 0;
    cudaError_t e = g->d.precision == CRN_FP64
                        ? launch_residual_fp64(g, (const double*)u, (double*)r, nullptr, nullptr, st, &nl)
                        : launch_residual_fp32(g, (const float*)u, (float*)r, nullptr, nullptr, st, &nl);
    launches += nl;
    ++evals;
    if (err == cudaSuccess) err = e;
  }
  int mode = 0;  // 0: y - J(dtau . y) (pseudo-time step), 1: J^T (dtau . y) (adjoint)
  int precond = 0;  // mode 0: 0 scales by dtau, 1 solves the radial line preconditioner
  bool ashift = false;  // mode 1: the shifted operator (D - J^T) P^-1 y of the pseudo-time adjoint

  // w->line: dinv, diag, lower, upper (forward: lower, diag, upper in slots 2,
  // 1, 3; adjoint: the transposed lines in slots 0, 1, 5); the Thomas factors
  // c_k in slot 4 and 1/m_k in slot 6 (line_factor)
  void line_factor() {
    double* L = w->line;
    const unsigned nb = (unsigned)((g->shape.nt * (int64_t)g->shape.np + NKB - 1) / NKB);
    if (mode == 1)
      line_factor_kernel<<<nb, NKB, 0, st>>>(g->shape, L, L + N, L + 5 * N, L + 4 * N, L + 6 * N);
    else
      line_factor_kernel<<<nb, NKB, 0, st>>>(g->shape, L + 2 * N, L + N, L + 3 * N, L + 4 * N, L + 6 * N);
    ++launches;
  }
  // z = P^-1 v (radial lines, from the factors)
  template <class TV>
  void line_solve(const TV* v, double* z) {
    const double* L = w->line;
    const unsigned nb = (unsigned)((NV * g->shape.nt * (int64_t)g->shape.np + NKB - 1) / NKB);
    line_solve_kernel<TV><<<nb, NKB, 0, st>>>(g->shape, mode == 1 ? L : L + 2 * N, L + 4 * N, L + 6 * N, v, z);
    ++launches;
  }

  // v: a Krylov vector (FP64, or FP32 with the FP32 basis, forward mode only)
  template <class TV>
  void apply(const TV* v, double* wout, const double* U, double b_rel, bool central) {
    if constexpr (sizeof(TV) == 8) {
      if (mode == 1) {
        adjoint_op(v, wout);
        return;
      }
    }
    apply_op(v, wout, U, b_rel, central);
  }

  // w_out = J^T (dtau . v) by the hand-written VJP of the residual; on FP32-bulk
  // grids ut holds the FP32 copy of U and the cotangent goes through rm / rt.
  // With ashift: w_out = (D - J^T) P^-1 v.
  void adjoint_op(const double* v, double* wout) {
    if (precond == 1) {
      line_solve(v, w->z);
    } else {
      precond_kernel<double><<<w->nblk, NKB, 0, st>>>(v, w->dtau, N, w->z, nullptr, nullptr, 0.0, w->part,
                                                      w->nblk, rows.minr, 0);
      ++launches;
    }
    vjp(w->z, wout);
    if (ashift) {
      shift_combine_kernel<<<grid, NKB, 0, st>>>(wout, w->z, w->dtau, N, n);
      ++launches;
    }
  }
  // w_out = J^T v (FP64 in and out)
  void vjp(const double* v, double* wout) {
    int nl = 0;
    cudaError_t e;
    if (g->d.precision == CRN_FP64) {
      e = launch_vjp_fp64(g, (const double*)w->ut, v, wout, nullptr, st, &nl);
    } else {
      perturb_kernel<float><<<grid, NKB, 0, st>>>(v, nullptr, nullptr, 0.0, n, (float*)w->rm);
      ++launches;
      e = launch_vjp_fp32(g, (const float*)w->ut, (const float*)w->rm, (float*)w->rt, nullptr, st, &nl);
      widen_kernel<<<grid, NKB, 0, st>>>((const float*)w->rt, n, wout);
      ++launches;
    }
    launches += nl;
    ++evals;
    if (err == cudaSuccess) err = e;
  }

  // w_out = v - J (dtau . v), J by a forward or central difference
  template <class TV>
  void apply_op(const TV* v, double* wout, const double* U, double b_rel, bool central) {
    if (precond == 1) {
      line_solve(v, w->z);
      precond_kernel<double><<<w->nblk, NKB, 0, st>>>(w->z, nullptr, N, w->z, U, w->out + rows.sumabs,
                                                      g->d.gamma - 1.0, w->part, w->nblk, rows.minr, 1);
    } else {
      precond_kernel<TV><<<w->nblk, NKB, 0, st>>>(v, w->dtau, N, w->z, U, w->out + rows.sumabs,
                                                  g->d.gamma - 1.0, w->part, w->nblk, rows.minr, 1);
    }
    ++launches;
    const double* dinv = precond == 1 ? w->line : nullptr;
    finish(rows.minr, 2, 2);
    eps_kernel<<<1, 1, 0, st>>>(w->out, rows.minr, rows.eps, b_rel);
    ++launches;
    const double* e = w->out + rows.eps;
    if (g->d.precision == CRN_FP64) {
      perturb_kernel<double><<<grid, NKB, 0, st>>>(U, w->z, e, 1.0, n, (double*)w->ut);
      ++launches;
      residual(w->ut, w->rt);
      const double* base = w->b;
      if (central) {
        perturb_kernel<double><<<grid, NKB, 0, st>>>(U, w->z, e, -1.0, n, (double*)w->ut);
        ++launches;
        residual(w->ut, w->rb);
        base = (const double*)w->rb;
      }
      jvp_combine_kernel<double, TV><<<grid, NKB, 0, st>>>(v, (const double*)w->rt, base, e,
                                                           central ? 2.0 : 1.0, n, wout, dinv, w->z, N);
    } else {
      perturb_kernel<float><<<grid, NKB, 0, st>>>(U, w->z, e, 1.0, n, (float*)w->ut);
      ++launches;
      residual(w->ut, w->rt);
      const float* base = (const float*)w->rb;
      if (central) {
        perturb_kernel<float><<<grid, NKB, 0, st>>>(U, w->z, e, -1.0, n, (float*)w->ut);
        ++launches;
        residual(w->ut, w->rm);
        base = (const float*)w->rm;
      }
      jvp_combine_kernel<float, TV><<<grid, NKB, 0, st>>>(v, (const float*)w->rt, base, e,
                                                          central ? 2.0 : 1.0, n, wout, dinv, w->z, N);
    }
    ++launches;
  }
};

// base residual b = R(U) (FP64) and, on FP32 grids, the FP32-bulk residual
// of the FP32 copy of U in rb (the base of forward differences); with
// outer64, b is the FP64 residual of the FP64 state instead of rb widened
void base_residual(Ctx& c, const double* U, bool outer64) {
  if (c.g->d.precision == CRN_FP64) {
    c.residual(U, c.w->b);
  } else {
    perturb_kernel<float><<<c.grid, NKB, 0, c.st>>>(U, nullptr, nullptr, 0.0, c.n, (float*)c.w->ut);
    ++c.launches;
    c.residual(c.w->ut, c.w->rb);
    if (outer64) {
      int nl = 0;
      const cudaError_t e = launch_residual_fp64(c.g, U, c.w->b, nullptr, nullptr, c.st, &nl);
      c.launches += nl;
      ++c.evals;
      if (c.err == cudaSuccess) c.err = e;
    } else {
      widen_kernel<<<c.grid, NKB, 0, c.st>>>((const float*)c.w->rb, c.n, c.w->b);
      ++c.launches;
    }
  }
}

// GMRES(m) with restarts on y -> y - J(dtau . y) for the right-hand side b;
// the solution y is left in w->x.  Returns the final relative residual.
double gmres(Ctx& c, const double* U, const crn_nk_options& o, double b_rel, double bnorm, int& iters) {
  const bool central = o.fd_central != 0;
  NkWork* w = c.w;
  const int m = o.krylov_dim;
  // FP32 basis (forward mode): V_j in Vf, the new Arnoldi vector in wf after
  // its FP64 product; FP64 basis: V_j and the new vector in V
  const bool f32 = c.mode == 0 && use_basis32(o) && w->Vf;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m), h(m + 1), h2(m + 1);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  // V_0 = r / beta from an FP64 vector r
  auto first = [&](const double* r, double beta) {
    if (f32) {
      c.to32(w->Vf, r, 1.0 / beta);
    } else {
      scale_kernel<<<c.grid, NKB, 0, c.st>>>(w->V, r, 1.0 / beta, c.n);
      ++c.launches;
    }
  };
  cudaMemsetAsync(w->x, 0, sizeof(double) * c.n, c.st);
  iters = 0;
  double rel = 1.0;
  if (!(bnorm > 0.0)) return 0.0;
  for (int cycle = 0; cycle <= o.max_restarts; ++cycle) {
    // r = b - A x; V_0 = r / |r|
    double beta;
    if (cycle == 0) {
      beta = bnorm;
      first(w->b, beta);
    } else {
      c.apply(w->x, w->w, U, b_rel, central);
      sub_kernel<<<c.grid, NKB, 0, c.st>>>(w->w, w->b, w->w, c.n);
      ++c.launches;
      beta = c.norm(w->w);
      if (!c.ok()) return rel;
      rel = beta / bnorm;
      if (rel <= o.lin_rtol || !(beta > 0.0)) return rel;
      first(w->w, beta);
    }
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double* vn = w->V + (size_t)(j + 1) * c.n;  // FP64 basis: the new vector in place
      float* vf = w->wf;                          // FP32 basis: the new vector
      if (f32) {
        c.apply(w->Vf + (size_t)j * c.n, w->w, U, b_rel, central);
        c.to32(vf, w->w, 1.0);
      } else {
        c.apply(w->V + (size_t)j * c.n, vn, U, b_rel, central);
      }
      ++iters;
      auto dots = [&](bool ww) { if (f32) c.dots32(j + 1, vf, ww); else c.dots(j + 1, vn, ww); };
      auto combine = [&](const double* coef) {
        if (f32) c.combine32(vf, coef, j + 1); else c.combine(vn, coef, j + 1);
      };
      auto norm = [&]() { return f32 ? c.norm32(vf) : c.norm(vn); };
      // classical Gram-Schmidt, repeated once if the norm dropped by > 0.7
      dots(true);
      c.fetch(0, j + 1);
      c.fetch(c.rows.ww, 1);
      if (!c.ok()) return rel;
      const double before = std::sqrt(std::max(w->host[c.rows.ww], 0.0));
      for (int t = 0; t <= j; ++t) h[t] = w->host[t];
      for (int t = 0; t <= j; ++t) h2[t] = -h[t];
      combine(h2.data());
      double after = norm();
      if (after < 0.7 * before) {
        dots(false);
        c.fetch(0, j + 1);
        if (!c.ok()) return rel;
        for (int t = 0; t <= j; ++t) { h2[t] = -w->host[t]; h[t] += w->host[t]; }
        combine(h2.data());
        after = norm();
      }
      if (!c.ok()) return rel;
      for (int t = 0; t <= j; ++t) Hat(t, j) = h[t];
      Hat(j + 1, j) = after;
      if (after > 0.0) {
        if (f32) {
          c.to32(w->Vf + (size_t)(j + 1) * c.n, vf, 1.0 / after);
        } else {
          scale_kernel<<<c.grid, NKB, 0, c.st>>>(vn, vn, 1.0 / after, c.n);
          ++c.launches;
        }
      }
      // Givens rotations on column j
      for (int t = 0; t < j; ++t) {
        const double a = Hat(t, j), bb = Hat(t + 1, j);
        Hat(t, j) = cs[t] * a + sn[t] * bb;
        Hat(t + 1, j) = -sn[t] * a + cs[t] * bb;
      }
      const double a = Hat(j, j), bb = Hat(j + 1, j);
      const double r = std::hypot(a, bb);
      cs[j] = r > 0.0 ? a / r : 1.0;
      sn[j] = r > 0.0 ? bb / r : 0.0;
      Hat(j, j) = r;
      Hat(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      jdone = j + 1;
      rel = std::fabs(gv[j + 1]) / bnorm;
      if (rel <= o.lin_rtol || !(after > 0.0)) break;
    }
    // y = H^-1 g (upper triangular), x += sum y_t V_t
    for (int t = jdone - 1; t >= 0; --t) {
      double s = gv[t];
      for (int q = t + 1; q < jdone; ++q) s -= Hat(t, q) * y[q];
      y[t] = Hat(t, t) != 0.0 ? s / Hat(t, t) : 0.0;
    }
    if (f32) c.combine_x32(w->x, y.data(), jdone);
    else c.combine(w->x, y.data(), jdone);
    if (rel <= o.lin_rtol) break;
  }
  return rel;
}

int read_flags(crn_grid* g, cudaStream_t st, int64_t& cell) {
  unsigned int flags = 0;
  unsigned long long bad = ~0ull;
  cudaError_t e = cudaMemcpyAsync(&flags, g->err_flags, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, g->err_cell, sizeof(bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->err_flags, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->err_cell, 0xff, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return -1;
  cell = flags ? (int64_t)bad : -1;
  return flags ? 1 : 0;
}

// relative step: about sqrt(unit roundoff) for a forward difference, its cube
// root for a central one, of the precision the residual runs in
double default_b(const crn_grid* g, bool central) {
  if (g->d.precision == CRN_FP64) return std::ldexp(1.0, central ? -17 : -26);
  return std::ldexp(1.0, central ? -8 : -12);
}

// one step: dU in w->z (unscaled by alpha), U updated by alpha dU
// (returns early, without solving or moving U, when |R(U)| <= stop_below)
int nk_step(crn_grid* g, double* U, double cfl, const crn_nk_options& o, crn_nk_stats* out,
            cudaStream_t st, int& launches, double stop_below, bool& stopped) {
  stopped = false;
  cudaError_t e = ensure_work(g, o.krylov_dim);
  if (e == cudaSuccess && use_basis32(o)) e = ensure_basis32(g->nk);
  if (e != cudaSuccess) return report(CRN_E_CUDA, std::string("Newton-Krylov workspace: ") + cudaGetErrorString(e));
  Ctx c(g, st);
  c.precond = o.precond;
  NkWork* w = c.w;
  const double b_rel = o.fd_rel > 0.0 ? o.fd_rel : default_b(g, o.fd_central != 0);
  const double gm1 = g->d.gamma - 1.0;
  int64_t bad_cell = -1;
  if (read_flags(g, st, bad_cell) < 0) return report(CRN_E_CUDA, "reading the error word");
  // local time steps, variable scales, R(U)
  {
    const Geo<double>& g64 = g->g64.geo;
    if (g->d.precision == CRN_FP64)
      local_dt_kernel<double><<<c.grid, NKB, 0, st>>>(g->shape, g64, g->d.gamma, g->d.c_h, U, cfl, w->dtau);
    else
      local_dt_kernel<float><<<c.grid, NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U, cfl, w->dtau);
    ++c.launches;
  }
  if (o.precond == 1) {
    double* L = w->line;
    if (g->d.precision == CRN_FP64)
      line_coef_kernel<double><<<c.grid, NKB, 0, st>>>(g->shape, g->g64.geo, g->d.gamma, g->d.c_h, U, cfl, L,
                                                       L + c.N, L + 2 * c.N, L + 3 * c.N);
    else
      line_coef_kernel<float><<<c.grid, NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U, cfl, L,
                                                      L + c.N, L + 2 * c.N, L + 3 * c.N);
    ++c.launches;
    c.line_factor();
  }
  absmean_kernel<<<w->nblk, NKB, 0, st>>>(U, c.N, w->part, w->nblk, c.rows.sumabs);
  ++c.launches;
  c.finish(c.rows.sumabs, NV, 0);
  const bool outer64 = g->d.precision == CRN_FP32_BULK && o.outer_fp64 != 0;
  if (outer64) {  // the FP64 tiled kernels' shared-memory opt-in (an FP32-bulk grid skips it)
    e = prepare_fp64();
    if (e != cudaSuccess) return report(CRN_E_CUDA, std::string("FP64 residual set-up: ") + cudaGetErrorString(e));
  }
  base_residual(c, U, outer64);
  const double bnorm = c.norm(w->b);
  if (!c.ok()) return report(CRN_E_CUDA, std::string("Newton-Krylov: ") + cudaGetErrorString(c.err));
  int flagged = read_flags(g, st, bad_cell);
  if (flagged) {
    g->last_bad_cell = bad_cell;
    launches += c.launches;
    char buf[160];
    std::snprintf(buf, sizeof(buf), "non-physical or non-finite state at cell %lld", (long long)bad_cell);
    return report(CRN_E_NONPHYSICAL, buf);
  }
  if (bnorm <= stop_below) {
    stopped = true;
    launches += c.launches;
    if (out) {
      out->res_l2 = bnorm;
      out->lin_rel = 0.0;
      out->alpha = 0.0;
      out->krylov_iters = 0;
      out->residual_evals = c.evals;
    }
    return CRN_OK;
  }
  int iters = 0;
  const double rel = gmres(c, U, o, b_rel, bnorm, iters);
  // dU = P^-1 y (dtau . y, or the radial line solve)
  if (o.precond == 1) {
    c.line_solve(w->x, w->z);
  } else {
    precond_kernel<double><<<w->nblk, NKB, 0, st>>>(w->x, w->dtau, c.N, w->z, U, w->out + c.rows.sumabs, gm1,
                                            w->part, w->nblk, c.rows.minr, 0);
    ++c.launches;
  }
  // step length: relative-change limiter, then positivity
  double alpha = 1.0;
  if (o.max_rel_change > 0.0) {
    relchange_kernel<<<w->nblk, NKB, 0, st>>>(U, w->z, c.N, gm1, w->part, w->nblk, c.rows.relmax);
    ++c.launches;
    c.finish(c.rows.relmax, 1, 1);
    c.fetch(c.rows.relmax, 1);
    const double r = w->host[c.rows.relmax];
    if (r > o.max_rel_change) alpha = o.max_rel_change / r;
  }
  int halvings = 0;
  for (;;) {
    badcount_kernel<<<w->nblk, NKB, 0, st>>>(U, w->z, alpha, c.N, gm1, w->part, w->nblk, c.rows.bad);
    ++c.launches;
    c.finish(c.rows.bad, 1, 0);
    c.fetch(c.rows.bad, 1);
    if (!c.ok()) break;
    if (w->host[c.rows.bad] == 0.0) break;
    if (++halvings > 40) { alpha = 0.0; break; }
    alpha *= 0.5;
  }
  if (alpha > 0.0) {
    apply_kernel<<<c.grid, NKB, 0, st>>>(U, w->z, alpha, c.n);
    ++c.launches;
  }
  if (!c.ok()) return report(CRN_E_CUDA, std::string("Newton-Krylov: ") + cudaGetErrorString(c.err));
  flagged = read_flags(g, st, bad_cell);  // a perturbed state of a JVP was non-physical
  launches += c.launches;
  if (out) {
    out->res_l2 = bnorm;
    out->lin_rel = rel;
    out->alpha = alpha;
    out->krylov_iters = iters;
    out->residual_evals = c.evals;
  }
  if (flagged) {
    g->last_bad_cell = bad_cell;
    return report(CRN_E_NONPHYSICAL, "a Jacobian-vector product met a non-physical perturbed state");
  }
  if (alpha == 0.0) return report(CRN_E_NONPHYSICAL, "no step length keeps rho and p positive");
  return CRN_OK;
}

int check_nk_options(const crn_nk_options& o) {
  if (o.krylov_dim < 1 || o.krylov_dim > 500) return report(CRN_E_ARG, "krylov_dim must be in [1, 500]");
  if (o.max_restarts < 0 || o.max_restarts > 1000) return report(CRN_E_ARG, "max_restarts must be in [0, 1000]");
  if (!(std::isfinite(o.lin_rtol) && o.lin_rtol > 0.0 && o.lin_rtol < 1.0))
    return report(CRN_E_ARG, "lin_rtol must be in (0, 1)");
  if (!(std::isfinite(o.fd_rel) && o.fd_rel >= 0.0 && o.fd_rel < 0.1))
    return report(CRN_E_ARG, "fd_rel must be in [0, 0.1)");
  if (!std::isfinite(o.max_rel_change)) return report(CRN_E_ARG, "max_rel_change must be finite");
  if (o.fd_central != 0 && o.fd_central != 1) return report(CRN_E_ARG, "fd_central must be 0 or 1");
  if (o.precond != 0 && o.precond != 1) return report(CRN_E_ARG, "precond must be 0 or 1");
  if (o.basis_fp32 < -1 || o.basis_fp32 > 1) return report(CRN_E_ARG, "basis_fp32 must be -1, 0 or 1");
  if (!(std::isfinite(o.adjoint_cfl) && o.adjoint_cfl >= 0.0)) return report(CRN_E_ARG, "adjoint_cfl must be >= 0");
  if (o.adjoint_outer < 1 || o.adjoint_outer > 100000) return report(CRN_E_ARG, "adjoint_outer must be in [1, 100000]");
  if (o.outer_fp64 != 0 && o.outer_fp64 != 1) return report(CRN_E_ARG, "outer_fp64 must be 0 or 1");
  if (o.adjoint_fgmres < 0 || o.adjoint_fgmres > 500) return report(CRN_E_ARG, "adjoint_fgmres must be in [0, 500]");
  return CRN_OK;
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_grid(crn_grid* g) {
  if (!g) return report(CRN_E_ARG, "grid is NULL");
  if (!g->have_br) return report(CRN_E_STATE, "crn_set_inner_boundary has not been called");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return report(CRN_E_ARG, "the current CUDA device is not the grid's device");
  return CRN_OK;
}

// adjoint solve J^T lambda = gbar at U (GMRES on J^T diag(dt), lambda = dt . y)
// and the sensitivity s = -(dR/dB_b)^T lambda
// (dR/dB_b)^T lambda into sens (negated: the sensitivity -(dR/dB_b)^T lambda),
// lambda in w->z, the state (or its FP32 copy) in w->ut
void sensitivity(Ctx& c, double* sens) {
  crn_grid* g = c.g;
  NkWork* w = c.w;
  int nl = 0;
  cudaError_t e;
  if (g->d.precision == CRN_FP64) {
    e = launch_vjp_fp64(g, (const double*)w->ut, w->z, w->w, sens, c.st, &nl);
  } else {
    perturb_kernel<float><<<c.grid, NKB, 0, c.st>>>(w->z, nullptr, nullptr, 0.0, c.n, (float*)w->rm);
    ++c.launches;
    e = launch_vjp_fp32(g, (const float*)w->ut, (const float*)w->rm, (float*)w->rt, sens, c.st, &nl);
  }
  c.launches += nl;
  ++c.evals;
  if (c.err == cudaSuccess) c.err = e;
  const int64_t nb = (int64_t)g->shape.nt * g->shape.np * (g->d.inner_bc == CRN_INNER_LARGE_E ? 2 : 1);
  scale_kernel<<<(unsigned)((nb + NKB - 1) / NKB), NKB, 0, c.st>>>(sens, sens, -1.0, nb);
  ++c.launches;
}

// Krylov acceleration of the pseudo-time adjoint: flexible GMRES(mf) on
// J^T lambda = gbar, right-preconditioned by one pass of the iteration, z =
// (J^T - D)^-1 v solved loosely like a pass (so the preconditioner changes from
// one application to the next: flexible GMRES keeps the directions z_j).  The
// passes damp the modes with |mu| >> D; the outer minimisation removes the few
// slow ones that the plain iteration contracts by d / (d - mu) ~ 1 per pass.
// lam and res (= gbar - J^T lam) on entry and exit; pass counts the
// preconditioner applications, kry their Krylov steps, rel the final true
// relative residual.
int adjoint_fgmres(Ctx& c, const double* U, const double* gbar, double* lam, double* res, double gnorm,
                   const crn_nk_options& inner, const crn_nk_options& o, int& pass, int& kry, double& rel) {
  NkWork* w = c.w;
  // FP32-bulk grids with outer_fp64: the outer products J^T z and the true
  // residual from the FP64 VJP of the FP64 state (the passes keep the FP32
  // VJP), so that the iteration converges past the FP32 VJP's rounding
  const bool outer64 = c.g->d.precision == CRN_FP32_BULK && o.outer_fp64 != 0;
  auto outer_vjp = [&](const double* v, double* wout) {
    if (!outer64) {
      c.vjp(v, wout);
      return;
    }
    int nl = 0;
    const cudaError_t e = launch_vjp_fp64(c.g, U, v, wout, nullptr, c.st, &nl);
    c.launches += nl;
    ++c.evals;
    if (c.err == cudaSuccess) c.err = e;
  };
  const int mf = std::min(o.adjoint_fgmres, o.krylov_dim);
  if (w->mf < mf) {
    cudaFree(w->fv);
    cudaFree(w->fz);
    w->fv = w->fz = nullptr;
    w->mf = 0;
    cudaError_t e = cudaMalloc(&w->fv, sizeof(double) * (size_t)(mf + 1) * c.n);
    if (e == cudaSuccess) e = cudaMalloc(&w->fz, sizeof(double) * (size_t)mf * c.n);
    if (e != cudaSuccess) {
      cudaFree(w->fv);
      cudaFree(w->fz);
      w->fv = w->fz = nullptr;
      return report(CRN_E_CUDA, std::string("adjoint FGMRES basis: ") + cudaGetErrorString(e));
    }
    w->mf = mf;
  }
  std::vector<double> H((size_t)(mf + 1) * mf), cs(mf), sn(mf), gv(mf + 1), y(mf), h(mf + 1), h2(mf + 1);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * mf + j]; };
  for (;;) {
    // the true residual of the current lambda
    if (pass > 0 || outer64) {
      outer_vjp(lam, w->w);
      sub_kernel<<<c.grid, NKB, 0, c.st>>>(res, gbar, w->w, c.n);
      ++c.launches;
    }
    const double beta = c.norm(res);
    if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
    rel = gnorm > 0.0 ? beta / gnorm : 0.0;
    if (!std::isfinite(rel)) return report(CRN_E_NONPHYSICAL, "the pseudo-time adjoint iteration diverged");
    if (!(rel > o.lin_rtol) || pass >= o.adjoint_outer) return CRN_OK;
    scale_kernel<<<c.grid, NKB, 0, c.st>>>(w->fv, res, 1.0 / beta, c.n);
    ++c.launches;
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    for (int j = 0; j < mf && pass < o.adjoint_outer; ++j) {
      double* vj = w->fv + (size_t)j * c.n;
      double* zj = w->fz + (size_t)j * c.n;
      double* vn = w->fv + (size_t)(j + 1) * c.n;
      // z_j = (J^T - D)^-1 v_j: the pass's loose solve of (D - J^T) z = -v_j (|v_j| = 1)
      scale_kernel<<<c.grid, NKB, 0, c.st>>>(w->b, vj, -1.0, c.n);
      ++c.launches;
      int it = 0;
      gmres(c, U, inner, 0.0, 1.0, it);
      kry += it;
      if (o.precond == 1) {
        c.line_solve(w->x, zj);
      } else {
        precond_kernel<double><<<w->nblk, NKB, 0, c.st>>>(w->x, w->dtau, c.N, zj, nullptr, nullptr, 0.0, w->part,
                                                          w->nblk, c.rows.minr, 0);
        ++c.launches;
      }
      ++pass;
      outer_vjp(zj, vn);  // J^T z_j
      // classical Gram-Schmidt against v_0 .. v_j, repeated once if the norm dropped by > 0.7
      c.dots_on(w->fv, j + 1, vn, true);
      c.fetch(0, j + 1);
      c.fetch(c.rows.ww, 1);
      if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
      const double before = std::sqrt(std::max(w->host[c.rows.ww], 0.0));
      for (int t = 0; t <= j; ++t) { h[t] = w->host[t]; h2[t] = -h[t]; }
      c.combine_on(vn, w->fv, h2.data(), j + 1);
      double after = c.norm(vn);
      if (after < 0.7 * before) {
        c.dots_on(w->fv, j + 1, vn, false);
        c.fetch(0, j + 1);
        if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
        for (int t = 0; t <= j; ++t) { h2[t] = -w->host[t]; h[t] += w->host[t]; }
        c.combine_on(vn, w->fv, h2.data(), j + 1);
        after = c.norm(vn);
      }
      if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
      for (int t = 0; t <= j; ++t) Hat(t, j) = h[t];
      Hat(j + 1, j) = after;
      if (after > 0.0) {
        scale_kernel<<<c.grid, NKB, 0, c.st>>>(vn, vn, 1.0 / after, c.n);
        ++c.launches;
      }
      for (int t = 0; t < j; ++t) {
        const double a = Hat(t, j), bb = Hat(t + 1, j);
        Hat(t, j) = cs[t] * a + sn[t] * bb;
        Hat(t + 1, j) = -sn[t] * a + cs[t] * bb;
      }
      const double a = Hat(j, j), bb = Hat(j + 1, j);
      const double r = std::hypot(a, bb);
      cs[j] = r > 0.0 ? a / r : 1.0;
      sn[j] = r > 0.0 ? bb / r : 0.0;
      Hat(j, j) = r;
      Hat(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      jdone = j + 1;
      if (std::fabs(gv[j + 1]) <= o.lin_rtol * gnorm || !(after > 0.0)) break;
    }
    // lambda += sum_t y_t z_t, y = H^-1 g
    for (int t = jdone - 1; t >= 0; --t) {
      double sm = gv[t];
      for (int q = t + 1; q < jdone; ++q) sm -= Hat(t, q) * y[q];
      y[t] = Hat(t, t) != 0.0 ? sm / Hat(t, t) : 0.0;
    }
    c.combine_on(lam, w->fz, y.data(), jdone);
    if (jdone == 0) return CRN_OK;
  }
}

// The adjoint by pseudo-time iteration, the counterpart of the primal's
// implicit steps: lambda <- lambda + delta with (D - J^T) delta ~= J^T lambda
// - gbar, D = diag(1 / (adjoint_cfl dt_c)), each correction solved loosely by
// GMRES (krylov_dim, relative tolerance 1e-1) on the shifted operator, right
// preconditioned by dtau or by the transposed radial lines of D - J.  The
// error of lambda contracts by D (D - mu)^-1 per pass for every eigenvalue mu
// of the (stable) J^T, where GMRES on J^T alone stagnates on large shells.
// Stops once |gbar - J^T lambda| <= lin_rtol |gbar| or after adjoint_outer
// passes.
int adjoint_pseudo_time(crn_grid* g, const double* U, const double* gbar, double* lambda, double* sens,
                        const crn_nk_options& o, crn_nk_stats* out, cudaStream_t st, int& launches) {
  cudaError_t e = ensure_work(g, o.krylov_dim);
  if (e == cudaSuccess && !g->vjp_buf && vjp_scratch_bytes(g) > 0)
    e = cudaMalloc(&g->vjp_buf, vjp_scratch_bytes(g));
  if (e == cudaSuccess && !g->nk->adj) e = cudaMalloc(&g->nk->adj, sizeof(double) * 2 * g->nk->n);
  if (e != cudaSuccess) return report(CRN_E_CUDA, std::string("adjoint workspace: ") + cudaGetErrorString(e));
  Ctx c(g, st);
  c.mode = 1;
  c.precond = o.precond;
  NkWork* w = c.w;
  double* lam = w->adj;
  double* res = w->adj + c.n;
  if (g->d.precision == CRN_FP64) {
    local_dt_kernel<double><<<c.grid, NKB, 0, st>>>(g->shape, g->g64.geo, g->d.gamma, g->d.c_h, U,
                                                    o.adjoint_cfl, w->dtau);
    cudaMemcpyAsync(w->ut, U, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  } else {
    local_dt_kernel<float><<<c.grid, NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U,
                                                   o.adjoint_cfl, w->dtau);
    perturb_kernel<float><<<c.grid, NKB, 0, st>>>(U, nullptr, nullptr, 0.0, c.n, (float*)w->ut);
    ++c.launches;
  }
  ++c.launches;
  if (o.precond == 1) {  // the radial lines of D - J at this CFL, transposed
    double* L = w->line;
    if (g->d.precision == CRN_FP64)
      line_coef_kernel<double><<<c.grid, NKB, 0, st>>>(g->shape, g->g64.geo, g->d.gamma, g->d.c_h, U,
                                                       o.adjoint_cfl, L, L + c.N, L + 2 * c.N, L + 3 * c.N);
    else
      line_coef_kernel<float><<<c.grid, NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U,
                                                      o.adjoint_cfl, L, L + c.N, L + 2 * c.N, L + 3 * c.N);
    line_transpose_kernel<<<c.grid, NKB, 0, st>>>(g->shape, L);  // writes the negated transposed lines
    negate_kernel<<<c.grid, NKB, 0, st>>>(L, c.N);
    negate_kernel<<<c.grid, NKB, 0, st>>>(L + 5 * c.N, c.N);
    c.launches += 4;
    c.line_factor();
  }
  cudaMemsetAsync(lam, 0, sizeof(double) * c.n, st);
  cudaMemcpyAsync(res, gbar, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  const double gnorm = c.norm(res);
  if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
  crn_nk_options inner = o;
  inner.max_restarts = 0;
  inner.lin_rtol = 1e-1;  // loose corrections: on 96x48x96 the outer-B_r adjoint needs half the
                          // Krylov steps of 1e-2 for the same passes (22 k against 42 k to 1e-6)
  int kry = 0, pass = 0;
  double rel = gnorm > 0.0 ? 1.0 : 0.0;
  c.ashift = true;
  if (o.adjoint_fgmres > 0) {
    const int rc = adjoint_fgmres(c, U, gbar, lam, res, gnorm, inner, o, pass, kry, rel);
    if (rc != CRN_OK) return rc;
  }
  for (; o.adjoint_fgmres == 0 && pass < o.adjoint_outer && rel > o.lin_rtol; ++pass) {
    if (pass > 0) {  // res = gbar - J^T lambda
      c.vjp(lam, w->w);
      sub_kernel<<<c.grid, NKB, 0, st>>>(res, gbar, w->w, c.n);
      ++c.launches;
      rel = c.norm(res) / gnorm;
      if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
      if (!(rel > o.lin_rtol)) break;
      if (!std::isfinite(rel)) return report(CRN_E_NONPHYSICAL, "the pseudo-time adjoint iteration diverged");
    }
    // (D - J^T) delta = -res, delta = P^-1 y
    scale_kernel<<<c.grid, NKB, 0, st>>>(w->b, res, -1.0, c.n);
    ++c.launches;
    int it = 0;
    gmres(c, U, inner, 0.0, rel * gnorm, it);
    kry += it;
    if (o.precond == 1) {
      c.line_solve(w->x, w->z);
    } else {
      precond_kernel<double><<<w->nblk, NKB, 0, st>>>(w->x, w->dtau, c.N, w->z, nullptr, nullptr, 0.0, w->part,
                                                      w->nblk, c.rows.minr, 0);
      ++c.launches;
    }
    add_kernel<<<c.grid, NKB, 0, st>>>(lam, w->z, c.n);
    ++c.launches;
  }
  c.ashift = false;
  cudaMemcpyAsync(w->z, lam, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  if (lambda) cudaMemcpyAsync(lambda, lam, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  if (sens && o.adjoint_fgmres > 0 && g->d.precision == CRN_FP32_BULK && o.outer_fp64 != 0) {
    // -(dR/dB_b)^T lambda from the FP64 VJP of the FP64 state, as the outer products
    int nl = 0;
    e = launch_vjp_fp64(g, U, lam, w->w, sens, st, &nl);
    c.launches += nl;
    ++c.evals;
    if (c.err == cudaSuccess) c.err = e;
    const int64_t nb = (int64_t)g->shape.nt * g->shape.np * (g->d.inner_bc == CRN_INNER_LARGE_E ? 2 : 1);
    scale_kernel<<<(unsigned)((nb + NKB - 1) / NKB), NKB, 0, st>>>(sens, sens, -1.0, nb);
    ++c.launches;
  } else if (sens) {
    sensitivity(c, sens);
  }
  if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
  launches += c.launches;
  if (out) {
    out->res_l2 = gnorm;
    out->lin_rel = rel;
    out->alpha = (double)pass;  // passes of the outer iteration
    out->krylov_iters = kry;
    out->residual_evals = c.evals;
  }
  return CRN_OK;
}

int adjoint_solve(crn_grid* g, const double* U, const double* gbar, double* lambda, double* sens,
                  const crn_nk_options& o, crn_nk_stats* out, cudaStream_t st, int& launches) {
  if (o.adjoint_cfl > 0.0) return adjoint_pseudo_time(g, U, gbar, lambda, sens, o, out, st, launches);
  cudaError_t e = ensure_work(g, o.krylov_dim);
  if (e == cudaSuccess && !g->vjp_buf && vjp_scratch_bytes(g) > 0)
    e = cudaMalloc(&g->vjp_buf, vjp_scratch_bytes(g));
  if (e != cudaSuccess) return report(CRN_E_CUDA, std::string("adjoint workspace: ") + cudaGetErrorString(e));
  Ctx c(g, st);
  c.mode = 1;
  c.precond = o.precond;
  NkWork* w = c.w;
  if (o.precond == 1) {
    double* L = w->line;
    if (g->d.precision == CRN_FP64)
      line_coef_kernel<double><<<c.grid, NKB, 0, st>>>(g->shape, g->g64.geo, g->d.gamma, g->d.c_h, U, INFINITY,
                                                       L, L + c.N, L + 2 * c.N, L + 3 * c.N);
    else
      line_coef_kernel<float><<<c.grid, NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U, INFINITY,
                                                      L, L + c.N, L + 2 * c.N, L + 3 * c.N);
    line_transpose_kernel<<<c.grid, NKB, 0, st>>>(g->shape, L);
    negate_kernel<<<c.grid, NKB, 0, st>>>(L + c.N, c.N);
    c.launches += 3;
    c.line_factor();
  }
  if (g->d.precision == CRN_FP64) {
    local_dt_kernel<double><<<c.grid, NKB, 0, st>>>(g->shape, g->g64.geo, g->d.gamma, g->d.c_h, U, 1.0, w->dtau);
    cudaMemcpyAsync(w->ut, U, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  } else {
    local_dt_kernel<float><<<c.grid, NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U, 1.0, w->dtau);
    perturb_kernel<float><<<c.grid, NKB, 0, st>>>(U, nullptr, nullptr, 0.0, c.n, (float*)w->ut);
    ++c.launches;
  }
  ++c.launches;
  cudaMemcpyAsync(w->b, gbar, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  const double bnorm = c.norm(w->b);
  if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
  int iters = 0;
  const double rel = gmres(c, U, o, 0.0, bnorm, iters);
  // lambda = P_a^-1 y (dt . y, or the transposed line solve)
  if (o.precond == 1) {
    c.line_solve(w->x, w->z);
  } else {
    precond_kernel<double><<<w->nblk, NKB, 0, st>>>(w->x, w->dtau, c.N, w->z, nullptr, nullptr, 0.0, w->part, w->nblk,
                                            c.rows.minr, 0);
    ++c.launches;
  }
  if (lambda) cudaMemcpyAsync(lambda, w->z, sizeof(double) * c.n, cudaMemcpyDeviceToDevice, st);
  if (sens) sensitivity(c, sens);  // (dR/dB_b)^T lambda from one more VJP, negated
  if (!c.ok()) return report(CRN_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(c.err));
  launches += c.launches;
  if (out) {
    out->res_l2 = bnorm;
    out->lin_rel = rel;
    out->alpha = 0.0;
    out->krylov_iters = iters;
    out->residual_evals = c.evals;
  }
  return CRN_OK;
}

}  // namespace
}  // namespace crn

extern "C" {

int crn_nk_options_default(crn_nk_options* o) {
  if (!o) return crn::report(CRN_E_ARG, "options pointer is NULL");
  std::memset(o, 0, sizeof(*o));
  o->krylov_dim = 30;
  o->max_restarts = 0;
  o->lin_rtol = 1e-3;
  o->fd_rel = 0.0;
  o->max_rel_change = 0.3;
  o->fd_central = 1;
  o->basis_fp32 = -1;
  o->adjoint_outer = 200;
  o->adjoint_cfl = 0.0;
  o->outer_fp64 = 1;
  o->adjoint_fgmres = 30;
  return CRN_OK;
}

int crn_steady_options_default(crn_steady_options* o) {
  if (!o) return crn::report(CRN_E_ARG, "options pointer is NULL");
  std::memset(o, 0, sizeof(*o));
  o->cfl0 = 2.0;
  o->cfl_max = 128.0;
  o->cfl_double_every = 10;
  o->max_steps = 500;
  o->tol_drop = 1e-6;
  return crn_nk_options_default(&o->nk);
}

int crn_local_dt(crn_grid* g, const double* U64_dev, double cfl, double* dtau_dev, void* stream) {
  if (!g) return crn::report(CRN_E_ARG, "grid is NULL");
  if (!U64_dev || !dtau_dev || !crn::device_ptr(U64_dev) || !crn::device_ptr(dtau_dev))
    return crn::report(CRN_E_ARG, "U64_dev and dtau_dev must be device pointers");
  if (!(std::isfinite(cfl) && cfl > 0.0)) return crn::report(CRN_E_ARG, "cfl must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = g->shape.ncell;
  const unsigned nb = (unsigned)std::min<int64_t>((N + crn::NKB - 1) / crn::NKB, (int64_t)g->cfg.num_sms * 16);
  if (g->d.precision == CRN_FP64)
    crn::local_dt_kernel<double><<<nb, crn::NKB, 0, st>>>(g->shape, g->g64.geo, g->d.gamma, g->d.c_h, U64_dev, cfl, dtau_dev);
  else
    crn::local_dt_kernel<float><<<nb, crn::NKB, 0, st>>>(g->shape, g->g32.geo, g->d.gamma, g->d.c_h, U64_dev, cfl, dtau_dev);
  g->last_launches = 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return crn::report(CRN_E_CUDA, std::string("crn_local_dt: ") + cudaGetErrorString(e));
  return CRN_OK;
}

int crn_newton_krylov_step(crn_grid* g, double* U64_dev, double cfl, const crn_nk_options* opt,
                           double* dU_dev, crn_nk_stats* stats, void* stream) {
  int rc = crn::check_grid(g);
  if (rc != CRN_OK) return rc;
  if (!U64_dev || !crn::device_ptr(U64_dev)) return crn::report(CRN_E_ARG, "U64_dev must be a device pointer");
  if (dU_dev && !crn::device_ptr(dU_dev)) return crn::report(CRN_E_ARG, "dU_dev must be a device pointer");
  if (!(std::isfinite(cfl) && cfl > 0.0)) return crn::report(CRN_E_ARG, "cfl must be finite and > 0");
  crn_nk_options o;
  if (opt) o = *opt; else crn_nk_options_default(&o);
  rc = crn::check_nk_options(o);
  if (rc != CRN_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int launches = 0;
  bool stopped = false;
  rc = crn::nk_step(g, U64_dev, cfl, o, stats, st, launches, -1.0, stopped);
  if (dU_dev && g->nk) {
    cudaError_t e = cudaMemcpyAsync(dU_dev, g->nk->z, sizeof(double) * 9 * g->shape.ncell,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess && rc == CRN_OK) rc = crn::report(CRN_E_CUDA, "copying dU");
  }
  g->last_launches = launches;
  return rc;
}

int crn_steady_solve(crn_grid* g, double* U64_dev, const crn_steady_options* opt, crn_steady_stats* stats,
                     double* history, int32_t history_len, void* stream) {
  int rc = crn::check_grid(g);
  if (rc != CRN_OK) return rc;
  if (!U64_dev || !crn::device_ptr(U64_dev)) return crn::report(CRN_E_ARG, "U64_dev must be a device pointer");
  crn_steady_options o;
  if (opt) o = *opt; else crn_steady_options_default(&o);
  if (!(std::isfinite(o.cfl0) && o.cfl0 > 0.0 && std::isfinite(o.cfl_max) && o.cfl_max >= o.cfl0))
    return crn::report(CRN_E_ARG, "need 0 < cfl0 <= cfl_max");
  if (o.cfl_double_every < 1 || o.max_steps < 0) return crn::report(CRN_E_ARG, "cfl_double_every >= 1, max_steps >= 0");
  if (!(std::isfinite(o.tol_drop) && o.tol_drop >= 0.0)) return crn::report(CRN_E_ARG, "tol_drop must be >= 0");
  rc = crn::check_nk_options(o.nk);
  if (rc != CRN_OK) return rc;
  if (history_len < 0 || (history_len > 0 && !history)) return crn::report(CRN_E_ARG, "history is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  crn_steady_stats s;
  std::memset(&s, 0, sizeof(s));
  double cfl = o.cfl0;
  int launches = 0;
  rc = CRN_OK;
  // each pass measures |R(U)| first; it stops there once the drop is reached
  // (or, after max_steps updates, to report the final residual)
  for (int step = 0;; ++step) {
    if (step > 0 && step % o.cfl_double_every == 0) cfl = std::min(2.0 * cfl, o.cfl_max);
    const double stop_below =
        step == o.max_steps ? INFINITY : (step == 0 ? -1.0 : o.tol_drop * s.res0);
    crn_nk_stats ns;
    std::memset(&ns, 0, sizeof(ns));
    bool stopped = false;
    rc = crn::nk_step(g, U64_dev, cfl, o.nk, &ns, st, launches, stop_below, stopped);
    if (step == 0) s.res0 = ns.res_l2;
    s.res_final = ns.res_l2;
    s.residual_evals += ns.residual_evals;
    s.krylov_iters += ns.krylov_iters;
    if (step < history_len) {
      history[4 * step + 0] = cfl;
      history[4 * step + 1] = ns.res_l2;
      history[4 * step + 2] = ns.alpha;
      history[4 * step + 3] = ns.krylov_iters;
    }
    if (rc != CRN_OK) break;
    if (stopped) {
      s.converged = ns.res_l2 <= o.tol_drop * s.res0 ? 1 : 0;
      break;
    }
    s.steps = step + 1;
  }
  g->last_launches = launches;
  if (stats) *stats = s;
  return rc;
}

int crn_adjoint_solve(crn_grid* g, const double* U64_dev, const double* gbar_dev, double* lambda_dev,
                      double* sens_dev, const crn_nk_options* opt, crn_nk_stats* stats, void* stream) {
  int rc = crn::check_grid(g);
  if (rc != CRN_OK) return rc;
  if (!U64_dev || !gbar_dev || !crn::device_ptr(U64_dev) || !crn::device_ptr(gbar_dev))
    return crn::report(CRN_E_ARG, "U64_dev and gbar_dev must be device pointers");
  if ((lambda_dev && !crn::device_ptr(lambda_dev)) || (sens_dev && !crn::device_ptr(sens_dev)))
    return crn::report(CRN_E_ARG, "lambda_dev and sens_dev must be device pointers");
  crn_nk_options o;
  if (opt) o = *opt; else crn_nk_options_default(&o);
  rc = crn::check_nk_options(o);
  if (rc != CRN_OK) return rc;
  int launches = 0;
  rc = crn::adjoint_solve(g, U64_dev, gbar_dev, lambda_dev, sens_dev, o, stats, (cudaStream_t)stream, launches);
  g->last_launches = launches;
  return rc;
}

}  // extern "C"
