// mhd_device.cuh -- device arithmetic of the MHD + GLM residual (sm_103a).
//
// Per-cell and per-face building blocks shared by the residual kernels:
// primitive recovery, the inner "low-E" and outer ghost states, the slope
// limiters, and the Rusanov + GLM face flux.  Templated on the arithmetic type
// T (double: the plain FP64 path; float: the FP32-bulk path).
//
// Paper: arXiv 2209.04481.  Equations of ideal MHD with gravity (Sect. 2.2) in
// Alfven-speed units; second-order FV with hyperbolic divergence cleaning
// (Sect. 2.1, cleaning speed c_h of Sect. 3.3); inner boundary of Sect. 3.2;
// outer boundary laws of Sect. 4.1 / Table 2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace crn {

// state indices: conservative (rho, mx, my, mz, bx, by, bz, E, psi) and
// primitive (rho, vx, vy, vz, bx, by, bz, p, psi) share positions 0, 4-6, 8.
constexpr int NV = 9;
// doubles per CTA in the reduction-partials array
constexpr int RED_STRIDE = 16;

// Geometry as 1D radial factors x per-column angular factors (all exact
// integrals of the shell, computed on the host in FP64):
//   |S_r(k face)|     = ra[k] * ar[j]          (ra = r^2)
//   |S_theta(j face)| = rb[k] * at[j face]     (rb = (r2^2 - r1^2) / 2)
//   |S_phi|           = rb[k] * dtheta
//   V(k, j)           = rv[k] * av[j]          (rv = (r2^3 - r1^3) / 3)
// Unit normals depend on (j, i) only.
template <class T>
struct Geo {
  const T* ra;      // [nr + 1]
  const T* rb;      // [nr]
  const T* rv;      // [nr]
  const T* inv_dm;  // [nr] 1 / (r_c(k) - r_c(k-1)), ghost centres mirrored
  const T* inv_dp;  // [nr] 1 / (r_c(k+1) - r_c(k))
  const T* hm;      // [nr] r_c(k) - r_f(k)
  const T* hp;      // [nr] r_f(k+1) - r_c(k)
  const T* grav;    // [nr] g0 / r_c(k)^2
  const T* ar;      // [nt]
  const T* at;      // [nt + 1] (0 at the poles)
  const T* av;      // [nt]
  const T* nr;      // [3][nt][np]      r-face unit normal
  const T* nth;     // [3][nt + 1][np]  theta-face unit normal
  const T* nph;     // [2][np]          phi-face unit normal (x, y; z = 0)
  const T* rhat;    // [3][nt][np]      radial unit vector at (theta_c, phi_c)
  T dtheta;
};

template <class T>
struct Phys {
  T gamma, gm1, igm1, ch, ch2, eps, rho_b, p_b;
  T fa, fb;        // outer ghost: rho, p and B_r factors (r_I / r_G)^a, ^b
  T fbp, fvr, fvp; // outer ghost: B_phi, V_r and V_phi factors
  T psi_out;       // outer ghost psi = psi_out * psi_I (-1: psi_b = 0, +1: zero-gradient)
  T psi_damp;      // GLM damping rate alpha: source -alpha psi in the psi equation (0: off)
  int inner_bc;    // inner boundary: 0 low-E, 1 large-E, 2 low-E with the V_r* magnitude
  double vr_star;  // large-E prescribed radial outflow
};

struct Shape {
  int nr, nt, np;
  int64_t ncell;
};

// (theta, phi) tile shapes of the ensemble kernel, all of 256 threads:
// tile t has ens_tt(t) x ens_tp(t) columns per CTA
constexpr int kEnsTileCount = 2;
__host__ __device__ constexpr int ens_tt(int t) { return t == 0 ? 8 : 16; }
__host__ __device__ constexpr int ens_tp(int t) { return t == 0 ? 32 : 16; }

template <class T> __device__ __forceinline__ T frcp(T x);
template <> __device__ __forceinline__ double frcp<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float frcp<float>(float x) { return __fdividef(1.0f, x); }
template <class T> __device__ __forceinline__ T fsqrt(T x);
template <> __device__ __forceinline__ double fsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float fsqrt<float>(float x) { return sqrtf(x); }

// ---------------------------------------------------------------------------
// primitive recovery [Sect. 2.2: E = p/(gamma-1) + rho V^2/2 + B^2/2]
// ---------------------------------------------------------------------------
// Threshold for the FP64 island of the FP32-bulk path: where B^2/2 exceeds the
// FP32 estimate of the internal energy (plasma beta < 2 (gamma-1) / gamma-ish),
// E - B^2/2 cancels and the internal energy is recomputed in FP64.
__device__ __forceinline__ void recover(const double (&u)[NV], const Phys<double>& ph,
                                        double (&w)[NV]) {
  const double ir = 1.0 / u[0];
  const double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  const double ek = 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz);
  const double eb = 0.5 * (u[4] * u[4] + u[5] * u[5] + u[6] * u[6]);
  w[0] = u[0];
  w[1] = vx; w[2] = vy; w[3] = vz;
  w[4] = u[4]; w[5] = u[5]; w[6] = u[6];
  w[7] = ph.gm1 * (u[7] - ek - eb);
  w[8] = u[8];
}

__device__ __forceinline__ void recover(const float (&u)[NV], const Phys<float>& ph,
                                        float (&w)[NV]) {
  const float ir = __fdividef(1.0f, u[0]);
  const float vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  const float ek = 0.5f * (u[1] * vx + u[2] * vy + u[3] * vz);
  const float eb = 0.5f * (u[4] * u[4] + u[5] * u[5] + u[6] * u[6]);
  float ei = u[7] - ek - eb;
  if (eb > ei) {
    // FP64 island: low-beta cell, E and B^2/2 nearly cancel
    const double bx = u[4], by = u[5], bz = u[6];
    const double e = (double)u[7] - 0.5 * (bx * bx + by * by + bz * bz) - (double)ek;
    ei = (float)e;
  }
  w[0] = u[0];
  w[1] = vx; w[2] = vy; w[3] = vz;
  w[4] = u[4]; w[5] = u[5]; w[6] = u[6];
  w[7] = ph.gm1 * ei;
  w[8] = u[8];
}

// ---------------------------------------------------------------------------
// ghost states (primitive); ghost = 2 * boundary - interior for V and B
// ---------------------------------------------------------------------------
// Inner boundary, Sect. 3.2 "low E": B_b = B_r rhat + tangential part of the
// interior B (Neumann in B_theta, B_phi); V_b = (V_I . B_b) B_b / |B_b|^2 so
// that V_b x B_b = 0; rho, p Dirichlet at the ghost centre; psi_b = 0
// (Sect. 3.3).  The vector algebra runs in FP64 in both precisions.
// Inner boundary, Sect. 3.2 "large E" (Wind-Predict): B_r and B_theta
// prescribed, B_phi Neumann; V_b = V_par (B_r rhat + B_theta thetahat) with
// V_par = V_r* B_r / (B_r^2 + B_theta^2), i.e. V_r = V_par B_r, V_theta =
// V_par B_theta, V_phi = 0; rho, p Dirichlet; psi_b = 0.  FP64.
template <class T>
__device__ __forceinline__ void large_e_ghost(const T (&wi)[NV], double br, double bt, double ex,
                                              double ey, double ez, const Phys<T>& ph, T (&wg)[NV]) {
  const double st = sqrt(ex * ex + ey * ey);        // sin(theta_c) > 0 at cell centres
  const double cp = ex / st, sp = ey / st;
  const double et[3] = {ez * cp, ez * sp, -st};     // thetahat
  const double ep[3] = {-sp, cp, 0.0};              // phihat
  const double er[3] = {ex, ey, ez};
  const double bip = (double)wi[4] * ep[0] + (double)wi[5] * ep[1];
  const double bpol2 = br * br + bt * bt;
  const double vpar = ph.vr_star * br / fmax(bpol2, 1e-300);
  wg[0] = ph.rho_b;
  wg[7] = ph.p_b;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double pol = br * er[c] + bt * et[c];
    wg[1 + c] = (T)(2.0 * vpar * pol - (double)wi[1 + c]);
    wg[4 + c] = (T)(2.0 * (pol + bip * ep[c]) - (double)wi[4 + c]);
  }
  wg[8] = -wi[8];
}

// The prescribed boundary field is read from br_plane[col] (B_r) and, for the
// large-E form, br_plane[nc + col] (B_theta).
template <class T>
__device__ __forceinline__ void inner_ghost_at(const T (&wi)[NV], const double* __restrict__ br_plane,
                                               int64_t col, int64_t nc, double ex, double ey,
                                               double ez, const Phys<T>& ph, T (&wg)[NV]);

template <class T>
__device__ __forceinline__ void inner_ghost(const T (&wi)[NV], double br, double ex, double ey,
                                            double ez, const Phys<T>& ph, T (&wg)[NV]) {
  const double bix = wi[4], biy = wi[5], biz = wi[6];
  const double vix = wi[1], viy = wi[2], viz = wi[3];
  const double bir = bix * ex + biy * ey + biz * ez;
  const double bbx = br * ex + (bix - bir * ex);
  const double bby = br * ey + (biy - bir * ey);
  const double bbz = br * ez + (biz - bir * ez);
  const double bb2 = bbx * bbx + bby * bby + bbz * bbz;
  // V_b = s B_b: s from the interior velocity (low-E) or from the prescribed
  // outflow, s = V_r* B_r / |B_b|^2 (low-E with the Wind-Predict magnitude)
  const double s = ph.inner_bc == 2 ? ph.vr_star * br / fmax(bb2, 1e-300)
                                    : (vix * bbx + viy * bby + viz * bbz) / fmax(bb2, 1e-300);
  wg[0] = ph.rho_b;
  wg[1] = (T)(2.0 * s * bbx - vix);
  wg[2] = (T)(2.0 * s * bby - viy);
  wg[3] = (T)(2.0 * s * bbz - viz);
  wg[4] = (T)(2.0 * bbx - bix);
  wg[5] = (T)(2.0 * bby - biy);
  wg[6] = (T)(2.0 * bbz - biz);
  wg[7] = ph.p_b;
  wg[8] = -wi[8];
}

template <class T>
__device__ __forceinline__ void inner_ghost_at(const T (&wi)[NV], const double* __restrict__ br_plane,
                                               int64_t col, int64_t nc, double ex, double ey,
                                               double ez, const Phys<T>& ph, T (&wg)[NV]) {
  if (ph.inner_bc == 1)
    large_e_ghost(wi, br_plane[col], br_plane[nc + col], ex, ey, ez, ph, wg);
  else
    inner_ghost(wi, br_plane[col], ex, ey, ez, ph, wg);
}

// Outer boundary, Sect. 4.1 / Table 2 (all nine cases) and Sect. 4.2: with
// s = r_I / r_G (r_G mirrors r_I about r_out): rho_G = rho_I s^a, p_G = p_I s^a,
// B_r,G = B_r,I s^b, B_phi,G = B_phi,I s^c, V_r,G = V_r,I s^(2-a) (if V_r r^2
// rho = const) or V_r,I, V_phi,G = V_phi,I s^e; theta components
// zero-gradient; psi_G = -psi_I (psi_b = 0) or psi_I.  The factors are in ph.
template <class T>
__device__ __forceinline__ void outer_ghost(const T (&wi)[NV], T ex, T ey, T ez,
                                            const Phys<T>& ph, T (&wg)[NV]) {
  const T st = sqrt(ex * ex + ey * ey);
  const T px = -ey / st, py = ex / st;  // phihat (z component 0)
  const T bir = wi[4] * ex + wi[5] * ey + wi[6] * ez;
  const T bip = wi[4] * px + wi[5] * py;
  const T vir = wi[1] * ex + wi[2] * ey + wi[3] * ez;
  const T vip = wi[1] * px + wi[2] * py;
  const T dbr = bir * ph.fb - bir, dbp = bip * ph.fbp - bip;
  const T dvr = vir * ph.fvr - vir, dvp = vip * ph.fvp - vip;
  wg[0] = wi[0] * ph.fa;
  wg[1] = wi[1] + dvr * ex + dvp * px;
  wg[2] = wi[2] + dvr * ey + dvp * py;
  wg[3] = wi[3] + dvr * ez;
  wg[4] = wi[4] + dbr * ex + dbp * px;
  wg[5] = wi[5] + dbr * ey + dbp * py;
  wg[6] = wi[6] + dbr * ez;
  wg[7] = wi[7] * ph.fa;
  wg[8] = ph.psi_out * wi[8];
}

// ---------------------------------------------------------------------------
// slope limiters on the two one-sided slopes a (backward), b (forward)
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T fmat(T a, T b, T c);
template <> __device__ __forceinline__ double fmat<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float fmat<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <int LIM, class T>
__device__ __forceinline__ T limited_slope(T a, T b, T eps) {
  if (LIM == 0) {  // unlimited central
    return (T)0.5 * (a + b);
  } else if (LIM == 1) {  // minmod
    if constexpr (sizeof(T) == 8) {
      // on the integer pipe (FP64 compares and products use the slow FP64
      // pipe): a b > 0 iff both are nonzero with equal sign bits, and the
      // magnitudes of non-negative doubles order as their bit patterns
      const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
      const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
      const unsigned long long ma = ba & 0x7fffffffffffffffull, mb = bb & 0x7fffffffffffffffull;
      const bool pos = ma != 0ull && mb != 0ull && ((ba ^ bb) >> 63) == 0ull;
      return pos ? (ma < mb ? a : b) : (T)0;
    } else {
      const T m = fabs(a) < fabs(b) ? a : b;
      return a * b > (T)0 ? m : (T)0;
    }
  } else {  // van Albada, smooth form: a (b^2 + eps) + b (a^2 + eps) is
            // (a + b)(a b + eps), one operation fewer; explicit FMAs so that
            // every kernel inlining this rounds it the same way
    const T num = (a + b) * fmat(a, b, eps);
    const T den = fmat(a, a, fmat(b, b, (T)2 * eps));
    return num * frcp(den);
  }
}

// Two limited slopes at once.  FP64 van Albada shares one division between
// them, 1/(d1 d2) times d2 and d1 (three multiplies and one IEEE division in
// place of two divisions on the slow FP64 pipe); d >= 2 eps > 0 and the
// slopes' squares keep d1 d2 far inside the binary64 range.  Every other case
// is two calls of limited_slope.
template <int LIM, class T>
__device__ __forceinline__ void limited_slope2(T a1, T b1, T a2, T b2, T eps, T& s1, T& s2) {
  if (LIM == 2 && sizeof(T) == 8) {
    const T n1 = (a1 + b1) * fmat(a1, b1, eps);
    const T d1 = fmat(a1, a1, fmat(b1, b1, (T)2 * eps));
    const T n2 = (a2 + b2) * fmat(a2, b2, eps);
    const T d2 = fmat(a2, a2, fmat(b2, b2, (T)2 * eps));
    const T inv = frcp(d1 * d2);
    s1 = n1 * (inv * d2);
    s2 = n2 * (inv * d1);
  } else {
    s1 = limited_slope<LIM>(a1, b1, eps);
    s2 = limited_slope<LIM>(a2, b2, eps);
  }
}

// ---------------------------------------------------------------------------
// Rusanov + GLM face flux through the unit normal n, times the face area.
// F* = (F(W_L) + F(W_R))/2 - lambda (U_R - U_L)/2,
// lambda = max(|u_n| + c_f over both sides, c_h);
// F_rho = rho u_n, F_m = rho V u_n + (p + B^2/2) n - B B_n,
// F_B = u_n B - B_n V + psi n, F_E = (E + p + B^2/2) u_n - B_n (V.B),
// F_psi = c_h^2 B_n.
// ---------------------------------------------------------------------------
template <class T>
struct Side {
  T un, bn, pt, en, sp;
};

template <class T>
__device__ __forceinline__ Side<T> side_terms(const T (&w)[NV], T nx, T ny, T nz,
                                               const Phys<T>& ph) {
  Side<T> s;
  const T ir = frcp(w[0]);
  s.un = w[1] * nx + w[2] * ny + w[3] * nz;
  s.bn = w[4] * nx + w[5] * ny + w[6] * nz;
  const T b2 = w[4] * w[4] + w[5] * w[5] + w[6] * w[6];
  const T v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  s.pt = w[7] + (T)0.5 * b2;
  s.en = w[7] * ph.igm1 + (T)0.5 * (w[0] * v2 + b2);
  const T a2 = ph.gamma * w[7] * ir;
  const T sum = a2 + b2 * ir;
  T disc = sum * sum - (T)4 * a2 * s.bn * s.bn * ir;
  disc = disc > (T)0 ? disc : (T)0;
  const T cf = fsqrt((T)0.5 * (sum + fsqrt(disc)));
  s.sp = fabs(s.un) + cf;
  return s;
}

template <class T>
__device__ __forceinline__ void rusanov(const T (&wl)[NV], const T (&wr)[NV], T nx, T ny, T nz,
                                        T area, const Phys<T>& ph, T (&f)[NV], T& lam_area) {
  const Side<T> L = side_terms(wl, nx, ny, nz, ph);
  const Side<T> R = side_terms(wr, nx, ny, nz, ph);
  T lam = L.sp > R.sp ? L.sp : R.sp;
  lam = lam > ph.ch ? lam : ph.ch;
  const T h = (T)0.5 * area;
  lam_area = lam * area;
  const T d = (T)0.5 * lam_area;  // halving is exact: the same value as (lam / 2) area
  // mass
  const T ml = wl[0] * L.un, mr = wr[0] * R.un;
  f[0] = h * (ml + mr) - d * (wr[0] - wl[0]);
  // momentum
  f[1] = h * ((ml * wl[1] + L.pt * nx - wl[4] * L.bn) + (mr * wr[1] + R.pt * nx - wr[4] * R.bn))
         - d * (wr[0] * wr[1] - wl[0] * wl[1]);
  f[2] = h * ((ml * wl[2] + L.pt * ny - wl[5] * L.bn) + (mr * wr[2] + R.pt * ny - wr[5] * R.bn))
         - d * (wr[0] * wr[2] - wl[0] * wl[2]);
  f[3] = h * ((ml * wl[3] + L.pt * nz - wl[6] * L.bn) + (mr * wr[3] + R.pt * nz - wr[6] * R.bn))
         - d * (wr[0] * wr[3] - wl[0] * wl[3]);
  // induction with the GLM gradient term
  f[4] = h * ((L.un * wl[4] - L.bn * wl[1] + wl[8] * nx) + (R.un * wr[4] - R.bn * wr[1] + wr[8] * nx))
         - d * (wr[4] - wl[4]);
  f[5] = h * ((L.un * wl[5] - L.bn * wl[2] + wl[8] * ny) + (R.un * wr[5] - R.bn * wr[2] + wr[8] * ny))
         - d * (wr[5] - wl[5]);
  f[6] = h * ((L.un * wl[6] - L.bn * wl[3] + wl[8] * nz) + (R.un * wr[6] - R.bn * wr[3] + wr[8] * nz))
         - d * (wr[6] - wl[6]);
  // energy
  const T vbl = wl[1] * wl[4] + wl[2] * wl[5] + wl[3] * wl[6];
  const T vbr = wr[1] * wr[4] + wr[2] * wr[5] + wr[3] * wr[6];
  f[7] = h * (((L.en + L.pt) * L.un - L.bn * vbl) + ((R.en + R.pt) * R.un - R.bn * vbr))
         - d * (R.en - L.en);
  // cleaning scalar
  f[8] = h * (ph.ch2 * (L.bn + R.bn)) - d * (wr[8] - wl[8]);
}

// across-pole / periodic mapping of a (possibly out-of-range) column (j, i):
// row -1 is row 0 and row -2 is row 1 on the opposite meridian (i + np/2),
// likewise beyond the south pole; phi is periodic.  Rows further out (only
// reached by the halo of a ragged tile, never by a used stencil) are clamped
// so that every mapped column is a valid index.
__device__ __forceinline__ void map_column(int& j, int& i, int nt, int np) {
  if (j < 0) { j = -1 - j; i += np / 2; }
  else if (j >= nt) { j = 2 * nt - 1 - j; i += np / 2; }
  j = j < 0 ? 0 : (j >= nt ? nt - 1 : j);
  while (i >= np) i -= np;  // i stays within a few periods: no integer division
  while (i < 0) i += np;
}

}  // namespace crn
