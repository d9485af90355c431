// vjp.cuh -- vector-Jacobian product of the residual: Ubar = (dR/dU)^T Rbar,
// Brbar = (dR/dB_r)^T Rbar.
//
// Reverse mode of the forward operator of residual.cuh, written by hand (the
// adjoint of every step: recovery, ghosts, limited reconstruction, the
// Rusanov + GLM flux, the accumulation and the gravity source), in two passes
// with recomputation instead of stored forward states:
//   vjp_faces  one thread per face: the cotangent of its flux x area,
//              fbar = Rbar_up / V_up - Rbar_lo / V_lo, is pulled back through
//              the flux and the reconstruction to the (up to) four stencil
//              cells' primitives; the 4 x 9 contributions are stored per face
//   vjp_cells  one thread per cell: gathers the contributions of every face
//              whose stencil holds the cell (in a fixed order, no atomics),
//              adds those that reached a ghost through the ghost's adjoint
//              (inner ghost: also into Brbar), then the adjoints of the
//              primitive recovery and of the gravity source.
// Non-smooth points follow the oracle's conventions: max(a, b) passes the
// derivative to a on a tie, d|x|/dx = +1 at 0, the clamp of the fast-speed
// discriminant at 0 has zero derivative.
#pragma once

#include "residual.cuh"

namespace crn {

// --------------------------------------------------------------------------
// limiter with its partial derivatives
// --------------------------------------------------------------------------
template <int LIM, class T>
__device__ __forceinline__ T slope_d(T a, T b, T eps, T& da, T& db) {
  if (LIM == 0) {
    da = (T)0.5; db = (T)0.5;
    return (T)0.5 * (a + b);
  } else if (LIM == 1) {
    if (!(a * b > (T)0)) { da = (T)0; db = (T)0; return (T)0; }
    if (fabs(a) < fabs(b)) { da = (T)1; db = (T)0; return a; }
    da = (T)0; db = (T)1;
    return b;
  } else {
    const T N = a * (b * b + eps) + b * (a * a + eps);
    const T D = a * a + b * b + (T)2 * eps;
    const T iD = (T)1 / D;
    const T s = N * iD;
    da = ((b * b + eps) + (T)2 * a * b - s * (T)2 * a) * iD;
    db = ((T)2 * a * b + (a * a + eps) - s * (T)2 * b) * iD;
    return s;
  }
}

// --------------------------------------------------------------------------
// adjoint of the Rusanov + GLM flux x area with respect to both face states
// --------------------------------------------------------------------------
template <class T>
struct SideFwd {
  T ir, un, bn, b2, v2, pt, en, a2, sum, sq, cf, sp, vb;
  bool clamp;
};

template <class T>
__device__ __forceinline__ SideFwd<T> side_fwd(const T (&w)[NV], T nx, T ny, T nz, const Phys<T>& ph) {
  SideFwd<T> s;
  s.ir = (T)1 / w[0];
  s.un = w[1] * nx + w[2] * ny + w[3] * nz;
  s.bn = w[4] * nx + w[5] * ny + w[6] * nz;
  s.b2 = w[4] * w[4] + w[5] * w[5] + w[6] * w[6];
  s.v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  s.vb = w[1] * w[4] + w[2] * w[5] + w[3] * w[6];
  s.pt = w[7] + (T)0.5 * s.b2;
  s.en = w[7] * ph.igm1 + (T)0.5 * (w[0] * s.v2 + s.b2);
  s.a2 = ph.gamma * w[7] * s.ir;
  s.sum = s.a2 + s.b2 * s.ir;
  T disc = s.sum * s.sum - (T)4 * s.a2 * s.bn * s.bn * s.ir;
  s.clamp = !(disc > (T)0);
  disc = s.clamp ? (T)0 : disc;
  s.sq = sqrt(disc);
  s.cf = sqrt((T)0.5 * (s.sum + s.sq));
  s.sp = fabs(s.un) + s.cf;
  return s;
}

// cotangent wb of one side's primitive state; sig = -1 (left) / +1 (right);
// spb = cotangent reaching this side's signal speed
template <class T>
__device__ __forceinline__ void side_adjoint(const T (&w)[NV], const SideFwd<T>& s, T nx, T ny, T nz,
                                             T h, T d, T sig, T spb, const Phys<T>& ph,
                                             const T (&fb)[NV], T (&wb)[NV]) {
  const T n[3] = {nx, ny, nz};
  const T rho = w[0];
  const T v[3] = {w[1], w[2], w[3]};
  const T b[3] = {w[4], w[5], w[6]};
  const T m = rho * s.un;
  const T ds = d * sig;
  T rhob = -ds * fb[0];
  T mb = h * fb[0];
  T vb[3], bb[3];
  T ptb = (T)0, bnb = (T)0, unb = (T)0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // momentum: h (m v_c + pt n_c - b_c bn) - d sig rho v_c
    mb += h * fb[1 + c] * v[c];
    rhob -= ds * fb[1 + c] * v[c];
    vb[c] = h * fb[1 + c] * m - ds * fb[1 + c] * rho;
    ptb += h * fb[1 + c] * n[c];
    bb[c] = -h * fb[1 + c] * s.bn;
    bnb -= h * fb[1 + c] * b[c];
    // induction: h (un b_c - bn v_c + psi n_c) - d sig b_c
    unb += h * fb[4 + c] * b[c];
    bb[c] += h * fb[4 + c] * s.un - ds * fb[4 + c];
    bnb -= h * fb[4 + c] * v[c];
    vb[c] -= h * fb[4 + c] * s.bn;
  }
  T psib = h * (fb[4] * nx + fb[5] * ny + fb[6] * nz);
  // energy: h ((en + pt) un - bn vb) - d sig en
  const T enb = h * fb[7] * s.un - ds * fb[7];
  ptb += h * fb[7] * s.un;
  unb += h * fb[7] * (s.en + s.pt);
  bnb -= h * fb[7] * s.vb;
  const T vbdb = -h * fb[7] * s.bn;
  // cleaning scalar: h ch^2 bn - d sig psi
  bnb += h * ph.ch2 * fb[8];
  psib -= ds * fb[8];
  // m = rho un
  rhob += mb * s.un;
  unb += mb * rho;
  // en = p igm1 + (rho v2 + b2) / 2, pt = p + b2 / 2, vb = v.b
  T pb = enb * ph.igm1 + ptb;
  rhob += (T)0.5 * enb * s.v2;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vb[c] += vbdb * b[c] + enb * rho * v[c];
    bb[c] += vbdb * v[c] + (enb + ptb) * b[c];
  }
  // signal speed sp = |un| + cf
  if (spb != (T)0) {
    unb += s.un >= (T)0 ? spb : -spb;
    const T qb = spb / ((T)2 * s.cf);        // cf = sqrt(q), q = (sum + sq) / 2
    T sumb = (T)0.5 * qb;
    const T sqb = (T)0.5 * qb;
    const T discb = (s.clamp || !(s.sq > (T)0)) ? (T)0 : sqb / ((T)2 * s.sq);
    // disc = sum^2 - 4 a2 bn^2 ir
    sumb += (T)2 * s.sum * discb;
    T a2b = -(T)4 * s.bn * s.bn * s.ir * discb;
    bnb -= (T)8 * s.a2 * s.bn * s.ir * discb;
    T irb = -(T)4 * s.a2 * s.bn * s.bn * discb;
    // sum = a2 + b2 ir
    a2b += sumb;
    const T b2b = sumb * s.ir;
    irb += sumb * s.b2;
    // a2 = gamma p ir
    pb += ph.gamma * s.ir * a2b;
    irb += ph.gamma * w[7] * a2b;
#pragma unroll
    for (int c = 0; c < 3; ++c) bb[c] += (T)2 * b[c] * b2b;
    rhob -= s.ir * s.ir * irb;
  }
  // un = v.n, bn = b.n
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vb[c] += unb * n[c];
    bb[c] += bnb * n[c];
  }
  wb[0] = rhob;
  wb[1] = vb[0]; wb[2] = vb[1]; wb[3] = vb[2];
  wb[4] = bb[0]; wb[5] = bb[1]; wb[6] = bb[2];
  wb[7] = pb;
  wb[8] = psib;
}

template <class T>
__device__ void rusanov_adjoint(const T (&wl)[NV], const T (&wr)[NV], T nx, T ny, T nz, T area,
                                const Phys<T>& ph, const T (&fb)[NV], T (&wlb)[NV], T (&wrb)[NV]) {
  const SideFwd<T> L = side_fwd(wl, nx, ny, nz, ph);
  const SideFwd<T> R = side_fwd(wr, nx, ny, nz, ph);
  // lambda = max(max(sp_L, sp_R), c_h); a tie passes the derivative to the first argument
  const bool selR = R.sp > L.sp;
  const T lam_s = selR ? R.sp : L.sp;
  const bool useC = ph.ch > lam_s;
  const T lam = useC ? ph.ch : lam_s;
  const T h = (T)0.5 * area, d = (T)0.5 * lam * area;
  // lambda cotangent: f_v contains -lambda area (U_R - U_L)_v / 2
  const T dU[NV] = {wr[0] - wl[0],
                    wr[0] * wr[1] - wl[0] * wl[1],
                    wr[0] * wr[2] - wl[0] * wl[2],
                    wr[0] * wr[3] - wl[0] * wl[3],
                    wr[4] - wl[4], wr[5] - wl[5], wr[6] - wl[6],
                    R.en - L.en, wr[8] - wl[8]};
  T lamb = (T)0;
#pragma unroll
  for (int v = 0; v < NV; ++v) lamb -= (T)0.5 * area * fb[v] * dU[v];
  const T spbL = (!useC && !selR) ? lamb : (T)0;
  const T spbR = (!useC && selR) ? lamb : (T)0;
  side_adjoint(wl, L, nx, ny, nz, h, d, (T)-1, spbL, ph, fb, wlb);
  side_adjoint(wr, R, nx, ny, nz, h, d, (T)1, spbR, ph, fb, wrb);
}

// --------------------------------------------------------------------------
// adjoints of the ghost maps and of the primitive recovery
// --------------------------------------------------------------------------
// inner low-E ghost: from the ghost's cotangent gb, add to the interior
// primitive's cotangent wib and return the cotangent of the prescribed B_r
template <class T>
__device__ double inner_ghost_adjoint(const T (&wi)[NV], double br, double ex, double ey, double ez,
                                      const Phys<T>& ph, const T (&gb)[NV], T (&wib)[NV]) {
  const double e[3] = {ex, ey, ez};
  const double bi[3] = {wi[4], wi[5], wi[6]};
  const double vi[3] = {wi[1], wi[2], wi[3]};
  const double bir = bi[0] * ex + bi[1] * ey + bi[2] * ez;
  double bbd[3];
  for (int c = 0; c < 3; ++c) bbd[c] = br * e[c] + (bi[c] - bir * e[c]);
  const double bb2 = bbd[0] * bbd[0] + bbd[1] * bbd[1] + bbd[2] * bbd[2];
  const bool wp = ph.inner_bc == 2;
  const double num = wp ? ph.vr_star * br : vi[0] * bbd[0] + vi[1] * bbd[1] + vi[2] * bbd[2];
  const bool floor = !(bb2 > 1e-300);
  const double den = floor ? 1e-300 : bb2;
  const double s = num / den;
  // ghost: V_g = 2 s B_b - V_I, B_g = 2 B_b - B_I, psi_g = -psi_I (rho, p fixed)
  double Bbb[3], sb = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double vgb = gb[1 + c], bgb = gb[4 + c];
    Bbb[c] = 2.0 * bgb + 2.0 * s * vgb;
    sb += 2.0 * vgb * bbd[c];
    wib[1 + c] -= (T)vgb;
    wib[4 + c] -= (T)bgb;
  }
  wib[8] -= gb[8];
  // s = num / den; num = V_I . B_b (low-E) or V_r* B_r (Wind-Predict magnitude)
  const double numb = sb / den;
  const double bb2b = floor ? 0.0 : -sb * s / den;
  double brb = 0.0;
  for (int c = 0; c < 3; ++c) Bbb[c] += 2.0 * bb2b * bbd[c];
  if (wp) {
    brb = numb * ph.vr_star;
  } else {
    for (int c = 0; c < 3; ++c) {
      wib[1 + c] += (T)(numb * bbd[c]);
      Bbb[c] += numb * vi[c];
    }
  }
  // B_b = B_r e + B_I - (B_I . e) e
  const double Be = Bbb[0] * ex + Bbb[1] * ey + Bbb[2] * ez;
  for (int c = 0; c < 3; ++c) wib[4 + c] += (T)(Bbb[c] - Be * e[c]);
  return brb + Be;
}

// large-E inner ghost: cotangents to the interior primitive and to the
// prescribed (B_r, B_theta), returned in brb[0], brb[1]
template <class T>
__device__ void large_e_ghost_adjoint(double br, double bt, double ex, double ey, double ez,
                                      const Phys<T>& ph, const T (&gb)[NV], T (&wib)[NV],
                                      double (&brb)[2]) {
  const double st = sqrt(ex * ex + ey * ey);
  const double cp = ex / st, sp = ey / st;
  const double et[3] = {ez * cp, ez * sp, -st};
  const double ep[3] = {-sp, cp, 0.0};
  const double er[3] = {ex, ey, ez};
  const double D = br * br + bt * bt;
  const bool floor = !(D > 1e-300);
  const double Dd = floor ? 1e-300 : D;
  const double vpar = ph.vr_star * br / Dd;
  double polb[3], vparb = 0.0, bipb = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double vg = gb[1 + c], bg = gb[4 + c];
    const double pol = br * er[c] + bt * et[c];
    polb[c] = 2.0 * vpar * vg + 2.0 * bg;
    vparb += 2.0 * vg * pol;
    bipb += 2.0 * bg * ep[c];
    wib[1 + c] -= (T)vg;
    wib[4 + c] -= (T)bg;
  }
  wib[8] -= gb[8];
  for (int c = 0; c < 3; ++c) wib[4 + c] += (T)(bipb * ep[c]);
  brb[0] = polb[0] * er[0] + polb[1] * er[1] + polb[2] * er[2];
  brb[1] = polb[0] * et[0] + polb[1] * et[1] + polb[2] * et[2];
  // V_par = vr* B_r / D, D = B_r^2 + B_theta^2
  if (floor) {
    brb[0] += vparb * ph.vr_star / Dd;
  } else {
    brb[0] += vparb * (ph.vr_star / D - 2.0 * ph.vr_star * br * br / (D * D));
    brb[1] += vparb * (-2.0 * ph.vr_star * br * bt / (D * D));
  }
}

// generalized outer ghost (Table 2 laws): the ghost is a fixed linear map of
// the interior primitive state
template <class T>
__device__ __forceinline__ void outer_ghost_adjoint(T ex, T ey, T ez, const Phys<T>& ph,
                                                    const T (&gb)[NV], T (&wib)[NV]) {
  const T st = sqrt(ex * ex + ey * ey);
  const T px = -ey / st, py = ex / st;
  const T e[3] = {ex, ey, ez};
  const T pe[3] = {px, py, (T)0};
  wib[0] += ph.fa * gb[0];
  wib[7] += ph.fa * gb[7];
  const T bre = gb[4] * ex + gb[5] * ey + gb[6] * ez, bpe = gb[4] * px + gb[5] * py;
  const T vre = gb[1] * ex + gb[2] * ey + gb[3] * ez, vpe = gb[1] * px + gb[2] * py;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    wib[1 + c] += gb[1 + c] + (ph.fvr - (T)1) * vre * e[c] + (ph.fvp - (T)1) * vpe * pe[c];
    wib[4 + c] += gb[4 + c] + (ph.fb - (T)1) * bre * e[c] + (ph.fbp - (T)1) * bpe * pe[c];
  }
  wib[8] += ph.psi_out * gb[8];
}

// U -> W recovery adjoint (plain, no low-beta island: derivatives only)
template <class T>
__device__ __forceinline__ void recover_adjoint(const T (&u)[NV], const Phys<T>& ph,
                                                const T (&wb)[NV], T (&ub)[NV]) {
  const T ir = (T)1 / u[0];
  const T v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
  const T pb = wb[7] * ph.gm1;
  T u0 = wb[0] + pb * (T)0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u0 -= wb[1 + c] * v[c] * ir;
    ub[1 + c] = wb[1 + c] * ir - pb * v[c];
    ub[4 + c] = wb[4 + c] - pb * u[4 + c];
  }
  ub[0] = u0;
  ub[7] = pb;
  ub[8] = wb[8];
}

// --------------------------------------------------------------------------
// pass 1: faces
// --------------------------------------------------------------------------
// contribution buffer of one face family: [4 stencil positions][NV][nfaces]
// positions: 0 = LL, 1 = L, 2 = R, 3 = RR (along the face normal's axis)
template <class T>
struct VjpBufs {
  T* cr;  // r faces     (nr + 1) * nt * np
  T* ct;  // theta faces nr * (nt + 1) * np
  T* cp;  // phi faces   nr * nt * np
  T* W;   // primitives of every cell [NV][N], recovered once per VJP (FP64 grids;
          // null on FP32-bulk grids, whose cheap recovery is redone per stencil)
};

// pass 0: W = primitives of U (the same recovery as the forward kernels)
template <class T>
__global__ void __launch_bounds__(256)
vjp_prims(Shape sh, Phys<T> ph, const T* __restrict__ U, T* __restrict__ W) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= sh.ncell) return;
  T w[NV];
  load_recover(U, sh.ncell, c, ph, w);
#pragma unroll
  for (int v = 0; v < NV; ++v) W[v * sh.ncell + c] = w[v];
}

// primitive state of cell (k, j, i) from W, ghosts included (as cell_prim)
template <class T>
__device__ void cell_w(const Shape& sh, const Geo<T>& g, const Phys<T>& ph, const double* __restrict__ Br,
                       const T* __restrict__ W, int k, int j, int i, T (&w)[NV]) {
  map_column(j, i, sh.nt, sh.np);
  const int64_t col = (int64_t)j * sh.np + i;
  const int64_t cs = (int64_t)sh.nt * sh.np;
  const int kk = k < 0 ? 0 : (k >= sh.nr ? sh.nr - 1 : k);
  T wi[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) wi[v] = W[v * sh.ncell + (int64_t)kk * cs + col];
  if (k < 0) {
    inner_ghost_at(wi, Br, col, cs, (double)g.rhat[col], (double)g.rhat[cs + col],
                   (double)g.rhat[2 * cs + col], ph, w);
  } else if (k >= sh.nr) {
    outer_ghost(wi, g.rhat[col], g.rhat[cs + col], g.rhat[2 * cs + col], ph, w);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = wi[v];
  }
}

template <class T>
__device__ __forceinline__ void put_contrib(T* buf, int64_t nf, int64_t f, int pos, const T (&c)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) buf[((int64_t)pos * NV + v) * nf + f] = c[v];
}

template <class T>
__device__ __forceinline__ void zero_contrib(T* buf, int64_t nf, int64_t f) {
  for (int q = 0; q < 4 * NV; ++q) buf[(int64_t)q * nf + f] = (T)0;
}

// One launch over the faces of all three axes (r faces, then theta, then
// phi): a thread per face, so that small grids still fill the GPU with
// several waves of these long threads.
template <class T, int LIM>
__global__ void __launch_bounds__(128)
vjp_faces(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br, const T* __restrict__ U,
          const T* __restrict__ Rb, VjpBufs<T> out) {
  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t cs = (int64_t)nt * np, N = sh.ncell;
  const int64_t nf0 = (int64_t)(nr + 1) * cs, nf1 = (int64_t)nr * (nt + 1) * np, nf2 = (int64_t)nr * cs;
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int axis = 0;  // 0 = r, 1 = theta, 2 = phi
  int64_t nf = nf0;
  T* buf = out.cr;
  if (f >= nf0) {
    f -= nf0;
    axis = 1; nf = nf1; buf = out.ct;
    if (f >= nf1) {
      f -= nf1;
      axis = 2; nf = nf2; buf = out.cp;
      if (f >= nf2) return;
    }
  }
  const T one = (T)1, half = (T)0.5;
  int k, j, i, a;           // a: face index along the axis; (k, j, i) the other two + dummy
  T nx, ny, nz, area;
  int lo[3], up[3];         // lower / upper cell (k, j, i)
  bool lo_in, up_in, first_order;
  if (axis == 0) {
    i = (int)(f % np); j = (int)((f / np) % nt); a = (int)(f / cs);
    lo[0] = a - 1; lo[1] = j; lo[2] = i; up[0] = a; up[1] = j; up[2] = i;
    lo_in = a >= 1; up_in = a <= nr - 1; first_order = !(lo_in && up_in);
    const int64_t col = (int64_t)j * np + i;
    nx = g.nr[col]; ny = g.nr[cs + col]; nz = g.nr[2 * cs + col];
    area = g.ra[a] * g.ar[j];
  } else if (axis == 1) {
    i = (int)(f % np); a = (int)((f / np) % (nt + 1)); k = (int)(f / ((int64_t)(nt + 1) * np));
    if (a == 0 || a == nt) { zero_contrib(buf, nf, f); return; }  // poles: zero area
    lo[0] = k; lo[1] = a - 1; lo[2] = i; up[0] = k; up[1] = a; up[2] = i;
    lo_in = up_in = true; first_order = false;
    const int64_t ts = (int64_t)(nt + 1) * np, fc = (int64_t)a * np + i;
    nx = g.nth[fc]; ny = g.nth[ts + fc]; nz = g.nth[2 * ts + fc];
    area = g.rb[k] * g.at[a];
  } else {
    a = (int)(f % np); j = (int)((f / np) % nt); k = (int)(f / cs);
    lo[0] = k; lo[1] = j; lo[2] = a - 1; up[0] = k; up[1] = j; up[2] = a;
    lo_in = up_in = true; first_order = false;
    nx = g.nph[a]; ny = g.nph[np + a]; nz = (T)0;
    area = g.rb[k] * g.dtheta;
  }
  // cotangent of the face's flux x area
  T fb[NV];
  {
    T slo = (T)0, sup = (T)0;
    int64_t clo = 0, cup = 0;
    if (lo_in) {
      int jj = lo[1], ii = lo[2];
      map_column(jj, ii, nt, np);
      clo = (int64_t)lo[0] * cs + (int64_t)jj * np + ii;
      slo = one / (g.rv[lo[0]] * g.av[jj]);
    }
    if (up_in) {
      int jj = up[1], ii = up[2];
      map_column(jj, ii, nt, np);
      cup = (int64_t)up[0] * cs + (int64_t)jj * np + ii;
      sup = one / (g.rv[up[0]] * g.av[jj]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
      fb[v] = (up_in ? Rb[v * N + cup] * sup : (T)0) - (lo_in ? Rb[v * N + clo] * slo : (T)0);
  }
  // the stencil (primitives, with ghosts) and the face states
  T wl[NV], wr[NV], wll[NV], wrr[NV];
  auto cell = [&](const int (&c)[3], int shift, T (&w)[NV]) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[axis] += shift;
    if (out.W)
      cell_w(sh, g, ph, Br, out.W, cc[0], cc[1], cc[2], w);
    else
      cell_prim(sh, g, ph, Br, U, cc[0], cc[1], cc[2], w);
  };
  cell(lo, 0, wl);
  cell(up, 0, wr);
  T sl[NV], dla[NV], dlb[NV], sr[NV], dra[NV], drb[NV];
  T im_l = one, ip_l = one, hl = half, im_r = one, ip_r = one, hr = half;
  T fl_state[NV], fr_state[NV];
  if (first_order) {
#pragma unroll
    for (int v = 0; v < NV; ++v) { fl_state[v] = wl[v]; fr_state[v] = wr[v]; }
  } else {
    cell(lo, -1, wll);
    cell(up, 1, wrr);
    if (axis == 0) {
      const int kl = lo[0], ku = up[0];
      im_l = g.inv_dm[kl]; ip_l = g.inv_dp[kl]; hl = g.hp[kl];
      im_r = g.inv_dm[ku]; ip_r = g.inv_dp[ku]; hr = g.hm[ku];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T dd = wr[v] - wl[v];
      sl[v] = slope_d<LIM>((wl[v] - wll[v]) * im_l, dd * ip_l, ph.eps, dla[v], dlb[v]);
      sr[v] = slope_d<LIM>(dd * im_r, (wrr[v] - wr[v]) * ip_r, ph.eps, dra[v], drb[v]);
      fl_state[v] = wl[v] + sl[v] * hl;
      fr_state[v] = wr[v] - sr[v] * hr;
    }
  }
  T wlb[NV], wrb[NV];
  rusanov_adjoint(fl_state, fr_state, nx, ny, nz, area, ph, fb, wlb, wrb);
  T cLL[NV], cL[NV], cR[NV], cRR[NV];
  if (first_order) {
#pragma unroll
    for (int v = 0; v < NV; ++v) { cLL[v] = (T)0; cL[v] = wlb[v]; cR[v] = wrb[v]; cRR[v] = (T)0; }
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T tl = hl * wlb[v], tr = -hr * wrb[v];
      const T al = tl * dla[v], bl = tl * dlb[v], ar = tr * dra[v], br = tr * drb[v];
      cLL[v] = -im_l * al;
      cL[v] = wlb[v] + im_l * al - ip_l * bl - im_r * ar;
      cR[v] = wrb[v] + ip_l * bl + im_r * ar - ip_r * br;
      cRR[v] = ip_r * br;
    }
  }
  put_contrib(buf, nf, f, 0, cLL);
  put_contrib(buf, nf, f, 1, cL);
  put_contrib(buf, nf, f, 2, cR);
  put_contrib(buf, nf, f, 3, cRR);
}

// --------------------------------------------------------------------------
// pass 2: cells
// --------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void add_contrib(const T* buf, int64_t nf, int64_t f, int pos, T (&acc)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] += buf[((int64_t)pos * NV + v) * nf + f];
}

template <class T>
__global__ void __launch_bounds__(128)
vjp_cells(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br, const T* __restrict__ U,
          const T* __restrict__ Rb, VjpBufs<T> in, T* __restrict__ Ub, double* __restrict__ Brb) {
  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t cs = (int64_t)nt * np, N = sh.ncell;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int i = (int)(c % np), j = (int)((c / np) % nt), k = (int)(c / cs);
  const int64_t col = (int64_t)j * np + i;
  const int64_t nfr = (int64_t)(nr + 1) * cs, nft = (int64_t)nr * (nt + 1) * np, nfp = (int64_t)nr * cs;
  T wb[NV], gin[NV], gout[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { wb[v] = (T)0; gin[v] = (T)0; gout[v] = (T)0; }
  // ---- r faces: face index a = kf (between planes kf - 1 and kf)
  auto rface = [&](int kf) -> int64_t { return (int64_t)kf * cs + col; };
  // this cell as R of face k, L of face k + 1, RR of face k - 1, LL of face k + 2
  add_contrib(in.cr, nfr, rface(k), 2, wb);
  add_contrib(in.cr, nfr, rface(k + 1), 1, wb);
  if (k - 1 >= 0) add_contrib(in.cr, nfr, rface(k - 1), 3, wb);
  if (k + 2 <= nr) add_contrib(in.cr, nfr, rface(k + 2), 0, wb);
  if (k == 0) {  // inner ghost (plane -1): L of face 0, LL of face 1
    add_contrib(in.cr, nfr, rface(0), 1, gin);
    add_contrib(in.cr, nfr, rface(1), 0, gin);
  }
  if (k == nr - 1) {  // outer ghost (plane nr): R of face nr, RR of face nr - 1
    add_contrib(in.cr, nfr, rface(nr), 2, gout);
    add_contrib(in.cr, nfr, rface(nr - 1), 3, gout);
  }
  // ---- theta faces in this column: face index a = jf (rows jf - 1 | jf)
  auto tface = [&](int jf, int ii) -> int64_t { return ((int64_t)k * (nt + 1) + jf) * np + ii; };
  add_contrib(in.ct, nft, tface(j, i), 2, wb);
  add_contrib(in.ct, nft, tface(j + 1, i), 1, wb);
  if (j - 1 >= 0) add_contrib(in.ct, nft, tface(j - 1, i), 3, wb);
  if (j + 2 <= nt) add_contrib(in.ct, nft, tface(j + 2, i), 0, wb);
  // across the poles this cell is row -1 / row nt of the opposite column
  const int io = (i + np / 2) % np;
  if (j == 0) add_contrib(in.ct, nft, tface(1, io), 0, wb);
  if (j == nt - 1) add_contrib(in.ct, nft, tface(nt - 1, io), 3, wb);
  // ---- phi faces (periodic): face index a = if (cols if - 1 | if)
  auto pface = [&](int ifc) -> int64_t {
    ifc = (ifc % np + np) % np;
    return ((int64_t)k * nt + j) * np + ifc;
  };
  add_contrib(in.cp, nfp, pface(i), 2, wb);
  add_contrib(in.cp, nfp, pface(i + 1), 1, wb);
  add_contrib(in.cp, nfp, pface(i - 1), 3, wb);
  add_contrib(in.cp, nfp, pface(i + 2), 0, wb);
  // ---- ghosts
  T u[NV], w[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = U[v * N + c];
  recover(u, ph, w);
  if (k == 0) {
    const double ex = g.rhat[col], ey = g.rhat[cs + col], ez = g.rhat[2 * cs + col];
    if (ph.inner_bc == 1) {
      double brb[2];
      large_e_ghost_adjoint(Br[col], Br[cs + col], ex, ey, ez, ph, gin, wb, brb);
      if (Brb) { Brb[col] = brb[0]; Brb[cs + col] = brb[1]; }
    } else {
      const double brb = inner_ghost_adjoint(w, Br[col], ex, ey, ez, ph, gin, wb);
      if (Brb) Brb[col] = brb;
    }
  }
  if (k == nr - 1) outer_ghost_adjoint(g.rhat[col], g.rhat[cs + col], g.rhat[2 * cs + col], ph, gout, wb);
  // ---- recovery and gravity source
  T ub[NV];
  recover_adjoint(u, ph, wb, ub);
  const T gk = -g.grav[k];
  const T gx = gk * g.rhat[col], gy = gk * g.rhat[cs + col], gz = gk * g.rhat[2 * cs + col];
  // S_m = rho g, S_E = m . g
  ub[0] += Rb[1 * N + c] * gx + Rb[2 * N + c] * gy + Rb[3 * N + c] * gz;
  ub[1] += Rb[7 * N + c] * gx;
  ub[2] += Rb[7 * N + c] * gy;
  ub[3] += Rb[7 * N + c] * gz;
  ub[8] -= ph.psi_damp * Rb[8 * N + c];  // S_psi = -alpha psi
#pragma unroll
  for (int v = 0; v < NV; ++v) Ub[v * N + c] = ub[v];
}

}  // namespace crn
