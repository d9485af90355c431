// vjp_tiled.cuh -- the residual VJP, Ubar = (dR/dU)^T Rbar and
// Brbar = (dR/dB_r)^T Rbar, in two stencil-recomputing passes that keep every
// intermediate on chip (no per-face scratch in global memory).
//
// The reverse of the forward operator of residual.cuh (arXiv 2209.04481
// Sect. 2.1 limited reconstruction + Rusanov/GLM fluxes, Sect. 3.2 inner
// ghost, Sect. 4.1 outer ghost), split by axis.  With W the primitives, the
// face value of cell c on the side of face a is W_c +/- h s_c, s_c the limited
// slope L(a_c, b_c) of the one-sided differences a_c = (W_c - W_{c-1}) im_c,
// b_c = (W_{c+1} - W_c) ip_c.  The adjoint of one face gives the cotangents of
// its two face values (u_c of the upper value of the cell below, l_c of the
// lower value of the cell above); the slope's cotangent is
// sbar_c = hp_c u_c - hm_c l_c, and with abar = sbar dL/da, bbar = sbar dL/db
//     Wbar_c     += u_c + l_c + im_c abar_c - ip_c bbar_c
//     Wbar_{c-1} -= im_c abar_c,      Wbar_{c+1} += ip_c bbar_c.
// Every term reaching a cell comes from the faces at most 3/2 cells away.
//
//   vjp_radial   one CTA per block of 16 columns x 13 planes: the
//                primitives of planes k0 - 3 .. k0 + 15 (ghost planes built
//                by the forward ghost maps) and Rbar / V in shared memory;
//                one thread per r face k0 - 1 .. k0 + 14 (the faces that
//                reach the block's planes), then one per plane for its slope
//                adjoint, then one per own plane gathering its neighbours'
//                terms in a fixed order; the ghosts' cotangents go through
//                the ghost adjoints (inner: also into Brbar).  Writes the r
//                part of Wbar into Ubar.
//   vjp_lateral  one CTA per (theta, phi) tile of one plane: the primitives
//                of the tile and a 3-cell cross halo (theta arm: the tile's
//                columns, phi arm: its rows) and Rbar / V with a 2-cell halo
//                in shared memory; each cell's limited slope once, as the
//                face values of its faces; every theta and phi face that
//                reaches a tile cell gets its adjoint once, its cotangents
//                replacing its states; each cell then takes its slope
//                adjoints and the neighbours' terms are gathered in a fixed
//                order (no atomics); the r part is added, then the adjoints
//                of the primitive recovery and of the sources, in place in
//                Ubar.
//   Every load of a thread is issued before the first is used.
//
// Cells beyond a pole are the cells of the opposite column (Cartesian vector
// components need no change); a theta face beyond a pole is that column's
// face with the normal reversed, which keeps the Rusanov flux and its adjoint
// consistent: F(L, R, n) = -F(R, L, -n).
#pragma once

#include "vjp.cuh"

namespace crn {

// (j, i) of a cell up to three rows beyond a pole (two crossings when n_theta
// is 2): every crossing moves to the opposite column
__device__ __forceinline__ void map_column_far(int& j, int& i, int nt, int np) {
  // |j| stays below a tile height plus 3, so a few crossings suffice; the
  // clamp only guards the index
#pragma unroll 1
  for (int it = 0; it < 16 && (j < 0 || j >= nt); ++it) {
    j = j < 0 ? -1 - j : 2 * nt - 1 - j;
    i += np / 2;
  }
  j = j < 0 ? 0 : (j >= nt ? nt - 1 : j);
  while (i >= np) i -= np;
  while (i < 0) i += np;
}

// adjoint of the U -> W recovery written with the primitives W of the same
// cell (rho, V and B are W's own entries): as recover_adjoint
template <class T>
__device__ __forceinline__ void recover_adjoint_w(const T (&w)[NV], const Phys<T>& ph, const T (&wb)[NV],
                                                  T (&ub)[NV]) {
  const T ir = (T)1 / w[0];
  const T pb = wb[7] * ph.gm1;
  T u0 = wb[0] + pb * (T)0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u0 -= wb[1 + c] * w[1 + c] * ir;
    ub[1 + c] = wb[1 + c] * ir - pb * w[1 + c];
    ub[4 + c] = wb[4 + c] - pb * w[4 + c];
  }
  ub[0] = u0;
  ub[7] = pb;
  ub[8] = wb[8];
}

// --------------------------------------------------------------------------
// pass 1: the r faces of a block of RC columns x RK planes
// --------------------------------------------------------------------------
// Thread (f, c) takes r face k0 - 1 + f of column c0 + c: the faces that reach
// planes k0 .. k0 + RK - 1 are k0 - 1 .. k0 + RK + 1 (RK + 3 = RF of them), their
// stencils planes k0 - 3 .. k0 + RK + 2.  Then one thread per plane
// k0 - 1 .. k0 + RK takes that plane's slope adjoint, and one per own plane
// gathers the terms of its neighbours (and the ghost adjoints at the ends).
constexpr int RCOL = 16, RK = 13, RF = RK + 3;
constexpr int RWP = RK + 6;   // planes of primitives k0 - 3 .. k0 + RK + 2
constexpr int RRP = RK + 4;   // planes of Rbar / V and of the plane terms k0 - 2 .. k0 + RK + 1
static_assert(RF * RCOL == 256, "one r face per thread");

template <class T>
constexpr size_t radial_smem_bytes() {
  return sizeof(T) * ((size_t)NV * RWP * RCOL + (size_t)NV * RRP * RCOL + (size_t)2 * NV * RF * RCOL +
                      (size_t)3 * NV * RRP * RCOL);
}

template <class T, int LIM>
__global__ void __launch_bounds__(RF * RCOL, 2)
vjp_radial(Shape sh, Geo<T> g, Phys<T> ph, const double* __restrict__ Br, const T* __restrict__ U,
           const T* __restrict__ Rb, T* __restrict__ Wr, double* __restrict__ Brb) {
  extern __shared__ __align__(16) unsigned char rad_smem[];
  T* sW = reinterpret_cast<T*>(rad_smem);   // [NV][RWP][RCOL] primitives (ghost planes included)
  T* sR = sW + NV * RWP * RCOL;              // [NV][RRP][RCOL] Rbar / V
  T* sF = sR + NV * RRP * RCOL;              // [2][NV][RF][RCOL] face-value cotangents L, R
  T* sD = sF + 2 * NV * RF * RCOL;           // [NV][RRP][RCOL] a plane's own terms
  T* sXl = sD + NV * RRP * RCOL;             // [NV][RRP][RCOL] terms from the plane below
  T* sXh = sXl + NV * RRP * RCOL;            // [NV][RRP][RCOL] terms from the plane above

  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t cs = (int64_t)nt * np, N = sh.ncell;
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * RCOL;
  const int k0 = blockIdx.y * RK;
  const T zero = (T)0;
  auto wi = [&](int v, int p, int c) -> T& { return sW[(v * RWP + (p - (k0 - 3))) * RCOL + c]; };
  auto ri = [&](int v, int p, int c) -> T& { return sR[(v * RRP + (p - (k0 - 2))) * RCOL + c]; };
  auto pi = [&](T* a, int v, int p, int c) -> T& { return a[(v * RRP + (p - (k0 - 2))) * RCOL + c]; };

  // ---- primitives (ghosts included, zeros beyond them) and Rbar / V; every
  // load of a thread is issued before the first is used
  {
    constexpr int NT = RF * RCOL;
    constexpr int WPT = (RWP * RCOL + NT - 1) / NT, RPT = (RRP * RCOL + NT - 1) / NT;
    T uw[WPT][NV], ur[RPT][NV];
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
      const int q = tid + m * NT;
      const int c = q % RCOL, p = k0 - 3 + q / RCOL;
      const int64_t col = c0 + c;
      if (q < RWP * RCOL && col < cs && p >= -1 && p <= nr) {
        const int ps = p < 0 ? 0 : (p >= nr ? nr - 1 : p);   // a ghost is built from its interior cell
        load_raw(U, N, (int64_t)ps * cs + col, uw[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const int q = tid + m * NT;
      const int c = q % RCOL, p = k0 - 2 + q / RCOL;
      const int64_t col = c0 + c;
      if (q < RRP * RCOL && col < cs && p >= 0 && p < nr) load_raw(Rb + (int64_t)p * cs, N, col, ur[m]);
    }
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
      const int q = tid + m * NT;
      if (q >= RWP * RCOL) continue;
      const int c = q % RCOL, p = k0 - 3 + q / RCOL;
      const int64_t col = c0 + c;
      T w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = zero;
      if (col < cs && p >= -1 && p <= nr) {
        T wi0[NV];
        recover(uw[m], ph, wi0);
        if (p == -1) {
          inner_ghost_at(wi0, Br, col, cs, (double)g.rhat[col], (double)g.rhat[cs + col],
                         (double)g.rhat[2 * cs + col], ph, w);
        } else if (p == nr) {
          outer_ghost(wi0, g.rhat[col], g.rhat[cs + col], g.rhat[2 * cs + col], ph, w);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) w[v] = wi0[v];
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) wi(v, p, c) = w[v];
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const int q = tid + m * NT;
      if (q >= RRP * RCOL) continue;
      const int c = q % RCOL, p = k0 - 2 + q / RCOL;
      const int64_t col = c0 + c;
      const bool in = col < cs && p >= 0 && p < nr;
      const T sc = in ? (T)1 / (g.rv[p] * g.av[col / np]) : zero;
#pragma unroll
      for (int v = 0; v < NV; ++v) ri(v, p, c) = in ? ur[m][v] * sc : zero;
    }
  }
  __syncthreads();

  // ---- one r face per thread
  {
    const int f = tid / RCOL, c = tid % RCOL;
    const int a = k0 - 1 + f;
    const int64_t col = c0 + c;
    T wlb[NV], wrb[NV];
    if (col < cs && a >= 0 && a <= nr) {
      const bool fo = a == 0 || a == nr;  // boundary faces: first order
      T L[NV], R[NV], fb[NV];
      if (fo) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { L[v] = wi(v, a - 1, c); R[v] = wi(v, a, c); }
      } else {
        const T im1 = g.inv_dm[a - 1], ip1 = g.inv_dp[a - 1], hp1 = g.hp[a - 1];
        const T im0 = g.inv_dm[a], ip0 = g.inv_dp[a], hm0 = g.hm[a];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T w2 = wi(v, a - 2, c), w1 = wi(v, a - 1, c), w0 = wi(v, a, c), wp = wi(v, a + 1, c);
          T d0, d1;
          const T s1 = slope_d<LIM>((w1 - w2) * im1, (w0 - w1) * ip1, ph.eps, d0, d1);
          const T s0 = slope_d<LIM>((w0 - w1) * im0, (wp - w0) * ip0, ph.eps, d0, d1);
          L[v] = w1 + s1 * hp1;
          R[v] = w0 - s0 * hm0;
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) fb[v] = ri(v, a, c) - ri(v, a - 1, c);
      const int j = (int)(col / np);
      rusanov_adjoint(L, R, g.nr[col], g.nr[cs + col], g.nr[2 * cs + col], g.ra[a] * g.ar[j], ph, fb, wlb, wrb);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) { wlb[v] = zero; wrb[v] = zero; }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sF[(v * RF + f) * RCOL + c] = wlb[v];
      sF[((NV + v) * RF + f) * RCOL + c] = wrb[v];
    }
  }
  __syncthreads();
  // face a of column c: L cotangent, R cotangent
  auto fl = [&](int v, int a, int c) -> T { return sF[(v * RF + (a - (k0 - 1))) * RCOL + c]; };
  auto fr = [&](int v, int a, int c) -> T { return sF[((NV + v) * RF + (a - (k0 - 1))) * RCOL + c]; };

  // ---- slope adjoints of planes k0 - 1 .. k0 + RK: the upper value of plane
  // p feeds face p + 1 (unless first order), its lower value face p
  if (tid < (RK + 2) * RCOL) {
    const int c = tid % RCOL, p = k0 - 1 + tid / RCOL;
    if (c0 + c < cs && p >= 0 && p < nr) {
      const T im = g.inv_dm[p], ip = g.inv_dp[p], hp = g.hp[p], hm = g.hm[p];
      const bool up_fo = p + 1 == nr, lo_fo = p == 0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T ua = fl(v, p + 1, c), la = fr(v, p, c);   // direct cotangents (either order)
        const T ub = up_fo ? zero : ua, lb = lo_fo ? zero : la;
        const T sb = hp * ub - hm * lb;
        const T wm = wi(v, p - 1, c), w0 = wi(v, p, c), wq = wi(v, p + 1, c);
        T da, db;
        slope_d<LIM>((w0 - wm) * im, (wq - w0) * ip, ph.eps, da, db);
        const T A = im * sb * da, B = ip * sb * db;
        pi(sD, v, p, c) = ua + la + A - B;
        pi(sXh, v, p - 1, c) = -A;
        pi(sXl, v, p + 1, c) = B;
      }
    }
  }
  __syncthreads();

  // ---- own planes: gather, ghost adjoints, store the r part
  if (tid < RK * RCOL) {
    const int c = tid % RCOL, p = k0 + tid / RCOL;
    const int64_t col = c0 + c;
    if (col < cs && p < nr) {
      T b[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        b[v] = pi(sD, v, p, c);
        if (p >= 1) b[v] += pi(sXl, v, p, c);
        if (p <= nr - 2) b[v] += pi(sXh, v, p, c);
      }
      if (p == 0) {  // inner ghost (plane -1): face 0's L value and plane 0's slope
        T gb[NV], w0[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { gb[v] = fl(v, 0, c) + pi(sXh, v, -1, c); w0[v] = wi(v, 0, c); }
        const double ex = g.rhat[col], ey = g.rhat[cs + col], ez = g.rhat[2 * cs + col];
        if (ph.inner_bc == 1) {
          double bb[2];
          large_e_ghost_adjoint(Br[col], Br[cs + col], ex, ey, ez, ph, gb, b, bb);
          if (Brb) { Brb[col] = bb[0]; Brb[cs + col] = bb[1]; }
        } else {
          const double bb = inner_ghost_adjoint(w0, Br[col], ex, ey, ez, ph, gb, b);
          if (Brb) Brb[col] = bb;
        }
      }
      if (p == nr - 1) {  // outer ghost (plane nr): face nr's R value and plane nr - 1's slope
        T gb[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) gb[v] = fr(v, nr, c) + pi(sXl, v, nr, c);
        outer_ghost_adjoint(g.rhat[col], g.rhat[cs + col], g.rhat[2 * cs + col], ph, gb, b);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Wr[v * N + (int64_t)p * cs + col] = b[v];
    }
  }
}

// --------------------------------------------------------------------------
// pass 2: the theta and phi faces of one plane of a tile, then the cells
// --------------------------------------------------------------------------
template <int TT, int TP>
struct LatDims {
  static constexpr int NT = TT * TP;                  // threads = tile cells
  static constexpr int HT = TT + 6, HP = TP + 6;      // primitives: 3-cell halo
  static constexpr int RT = TT + 4, RP = TP + 4;      // Rbar / V: 2-cell halo
  static constexpr int NW = TT * HP + 6 * TP;         // cross positions (no corners)
  static constexpr int NR = TT * RP + 4 * TP;
  static constexpr int NFT = (TT + 3) * TP;           // theta faces j0 - 1 .. j0 + TT + 1
  static constexpr int NFP = TT * (TP + 3);           // phi faces i0 - 1 .. i0 + TP + 1
  static constexpr size_t elems() {
    return (size_t)NV * HT * HP + (size_t)NV * RT * RP + (size_t)2 * NV * (NFT + NFP) + (size_t)2 * NV * NT;
  }
  template <class T>
  static constexpr size_t smem_bytes() { return sizeof(T) * elems(); }
};

template <class T, int LIM, int TT, int TP, int MINB>
__global__ void __launch_bounds__(TT * TP, MINB)
vjp_lateral(Shape sh, Geo<T> g, Phys<T> ph, const T* __restrict__ U, const T* __restrict__ Rb,
            T* __restrict__ Ub) {
  using D = LatDims<TT, TP>;
  constexpr int NT = D::NT, HP = D::HP, HC = D::HT * D::HP, RP = D::RP, RC = D::RT * D::RP;
  constexpr int NFT = D::NFT, NFP = D::NFP;
  static_assert(NT % 32 == 0 && TT >= 2 && TP >= 2, "tile shape");
  extern __shared__ __align__(16) unsigned char lat_smem[];
  T* sW = reinterpret_cast<T*>(lat_smem);   // [NV][HT][HP] primitives
  T* sR = sW + NV * HC;                      // [NV][RT][RP] Rbar / V
  T* sFt = sR + NV * RC;                     // [2][NV][NFT] theta faces: L, R states, then their cotangents
  T* sFp = sFt + 2 * NV * NFT;               // [2][NV][NFP] phi faces, likewise
  T* sX = sFp + 2 * NV * NFP;                // [2][NV][NT]  neighbour terms (from below, from above)

  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t cs = (int64_t)nt * np, N = sh.ncell;
  const int tid = threadIdx.x;
  const int ntp = (np + TP - 1) / TP;
  const int j0 = (blockIdx.x / ntp) * TT, i0 = (blockIdx.x % ntp) * TP;
  const int k = blockIdx.y;
  if (k >= nr) return;
  const int jj = tid / TP, ii = tid % TP;
  const bool own = j0 + jj < nt && i0 + ii < np;
  const T zero = (T)0, half = (T)0.5;
  const T* Uk = U + (int64_t)k * cs;
  const T* Rk = Rb + (int64_t)k * cs;
  const T irv = (T)1 / g.rv[k];

  // ---- primitives of the cross (3-cell halo) and Rbar / V (2-cell halo):
  // every load of a thread is issued before the first is used (one round
  // trip to memory per CTA instead of one per cell)
  {
    constexpr int WPT = (D::NW + NT - 1) / NT, RPT = (D::NR + NT - 1) / NT;
    T uw[WPT][NV], ur[RPT][NV], rs[RPT];
    int ws[WPT], rsl[RPT];
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
      const int q = tid + m * NT;
      ws[m] = -1;
      if (q < D::NW) {
        int row, c;
        if (q < TT * HP) { row = 3 + q / HP; c = q % HP; }
        else { const int h = q - TT * HP; const int hr = h / TP; row = hr < 3 ? hr : TT + hr; c = 3 + h % TP; }
        int jg = j0 - 3 + row, ig = i0 - 3 + c;
        map_column_far(jg, ig, nt, np);
        ws[m] = row * HP + c;
        load_raw(Uk, N, (int64_t)jg * np + ig, uw[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const int q = tid + m * NT;
      rsl[m] = -1;
      if (q < D::NR) {
        int row, c;
        if (q < TT * RP) { row = 2 + q / RP; c = q % RP; }
        else { const int h = q - TT * RP; const int hr = h / TP; row = hr < 2 ? hr : TT + hr; c = 2 + h % TP; }
        int jg = j0 - 2 + row, ig = i0 - 2 + c;
        map_column_far(jg, ig, nt, np);
        rsl[m] = row * RP + c;
        rs[m] = g.av[jg];
        load_raw(Rk, N, (int64_t)jg * np + ig, ur[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
      if (ws[m] < 0) continue;
      T w[NV];
      recover(uw[m], ph, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) sW[v * HC + ws[m]] = w[v];
    }
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      if (rsl[m] < 0) continue;
      const T sc = irv / rs[m];
#pragma unroll
      for (int v = 0; v < NV; ++v) sR[v * RC + rsl[m]] = ur[m][v] * sc;
    }
  }
  __syncthreads();

  // ---- face values: every cell whose upper or lower value a face of the
  // tile needs takes its limited slope once (theta: rows j0 - 2 .. j0 + TT + 1
  // of the tile's columns; phi: columns i0 - 2 .. i0 + TP + 1 of its rows);
  // face f's L state goes to slot 0 of f, its R state to slot 1
  constexpr int NVT = (TT + 4) * TP, NVP = TT * (TP + 4);
  for (int q = tid; q < NVT + NVP; q += NT) {
    int wc, wstep, fup, flo, nf;   // fup / flo: face whose L / R state this cell gives (-1: none)
    T* F;
    if (q < NVT) {
      const int r = q / TP, c = q % TP;      // cell row j0 - 2 + r: frame row r + 1
      wc = (r + 1) * HP + c + 3; wstep = HP;
      fup = r < TT + 3 ? r * TP + c : -1;    // face above: row r
      flo = r >= 1 ? (r - 1) * TP + c : -1;  // face below: row r - 1
      F = sFt; nf = NFT;
    } else {
      const int qp = q - NVT;
      const int row = qp / (TP + 4), c = qp % (TP + 4);   // column i0 - 2 + c: frame col c + 1
      wc = (row + 3) * HP + c + 1; wstep = 1;
      fup = c < TP + 3 ? row * (TP + 3) + c : -1;
      flo = c >= 1 ? row * (TP + 3) + c - 1 : -1;
      F = sFp; nf = NFP;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* p = sW + v * HC + wc;
      const T wm = p[-wstep], w0 = p[0], wq = p[wstep];
      T d0, d1;
      const T sl = slope_d<LIM>(w0 - wm, wq - w0, ph.eps, d0, d1);
      if (fup >= 0) F[v * nf + fup] = w0 + half * sl;
      if (flo >= 0) F[(NV + v) * nf + flo] = w0 - half * sl;
    }
  }
  __syncthreads();

  // ---- face adjoints, theta faces first, then phi faces: the cotangents of
  // the face's L and R states replace them
  const T rbk = g.rb[k];
  for (int q = tid; q < NFT + NFP; q += NT) {
    T nx, ny, nz, area;
    bool live;
    int rlo, rstep;   // Rbar / V of the cells below and above: sR[rlo], sR[rlo + rstep]
    T* F;
    int fidx, nf;
    if (q < NFT) {
      const int fr = q / TP, c = q % TP;
      const int a = j0 - 1 + fr, ig = i0 + c;
      // faces that reach a tile cell: -1 .. nt + 1 (0 and nt are the poles)
      live = ig < np && a >= -1 && a <= nt + 1 && a != 0 && a != nt;
      if (live) {
        int af = a, ic = ig;
        T sgn = (T)1;
        if (a < 0 || a > nt) {    // beyond a pole: the opposite column's face, normal reversed
          af = a < 0 ? -a : 2 * nt - a;
          ic = ig + np / 2;
          ic = ic >= np ? ic - np : ic;
          sgn = (T)-1;
        }
        const int64_t ts = (int64_t)(nt + 1) * np, fc = (int64_t)af * np + ic;
        nx = sgn * g.nth[fc]; ny = sgn * g.nth[ts + fc]; nz = sgn * g.nth[2 * ts + fc];
        area = rbk * g.at[af];
      }
      rlo = fr * RP + (c + 2); rstep = RP;
      F = sFt; fidx = q; nf = NFT;
    } else {
      const int qp = q - NFT;
      const int row = qp / (TP + 3), fc = qp % (TP + 3);
      const int a = i0 - 1 + fc;
      live = j0 + row < nt && a <= np + 1;
      if (live) {
        const int am = a < 0 ? a + np : (a >= np ? a - np : a);
        nx = g.nph[am]; ny = g.nph[np + am]; nz = zero;
        area = rbk * g.dtheta;
      }
      rlo = (row + 2) * RP + fc; rstep = 1;
      F = sFp; fidx = qp; nf = NFP;
    }
    T wlb[NV], wrb[NV];
    if (live) {
      T L[NV], R[NV], fb[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        L[v] = F[v * nf + fidx];
        R[v] = F[(NV + v) * nf + fidx];
        fb[v] = sR[v * RC + rlo + rstep] - sR[v * RC + rlo];
      }
      rusanov_adjoint(L, R, nx, ny, nz, area, ph, fb, wlb, wrb);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) { wlb[v] = zero; wrb[v] = zero; }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      F[v * nf + fidx] = wlb[v];
      F[(NV + v) * nf + fidx] = wrb[v];
    }
  }
  __syncthreads();

  // the r part of this cell's cotangent and its Rbar for the sources: loads
  // issued now, used at the end
  const int jo = j0 + jj, io = i0 + ii;
  const int64_t colo = own ? (int64_t)jo * np + io : 0, cell = (int64_t)k * cs + colo;
  T wr[NV], rsrc[5];
  if (own) {
#pragma unroll
    for (int v = 0; v < NV; ++v) wr[v] = Ub[v * N + cell];
    rsrc[0] = __ldg(Rb + 1 * N + cell);
    rsrc[1] = __ldg(Rb + 2 * N + cell);
    rsrc[2] = __ldg(Rb + 3 * N + cell);
    rsrc[3] = __ldg(Rb + 7 * N + cell);
    rsrc[4] = __ldg(Rb + 8 * N + cell);
  }

  // ---- slope adjoints, theta then phi; neighbour terms through sX
  T acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = zero;
  T* xlo = sX;            // [NV][NT] term from the cell below (b-part of its slope)
  T* xhi = sX + NV * NT;  // [NV][NT] term from the cell above (a-part of its slope)
  // the slope adjoint of one cell: centre at sW[wc], neighbours at -/+ wstep;
  // face-value cotangents ub (upper) and lb (lower); returns the direct term
  // in dir and abar, bbar
  auto slope_adj = [&](int wc, int wstep, const T* F, int nf, int fu, int fl, T (&dir)[NV], T (&ab)[NV],
                       T (&bb)[NV]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* p = sW + v * HC + wc;
      const T wm = p[-wstep], w0 = p[0], wq = p[wstep];
      T da, db;
      slope_d<LIM>(w0 - wm, wq - w0, ph.eps, da, db);
      const T u = F[v * nf + fu], l = F[(NV + v) * nf + fl];
      const T sb = half * (u - l);
      ab[v] = sb * da;
      bb[v] = sb * db;
      dir[v] = u + l + ab[v] - bb[v];
    }
  };
  // one variable of it
  auto slope_adj1 = [&](int v, int wc, int wstep, const T* F, int nf, int fu, int fl, T& ab, T& bb) {
    const T* p = sW + v * HC + wc;
    const T wm = p[-wstep], w0 = p[0], wq = p[wstep];
    T da, db;
    slope_d<LIM>(w0 - wm, wq - w0, ph.eps, da, db);
    const T sb = half * (F[v * nf + fu] - F[(NV + v) * nf + fl]);
    ab = sb * da;
    bb = sb * db;
  };
  // the phi halo columns i0 - 1 and i0 + TP feed columns 0 and TP - 1: their
  // 2 TT x NV one-variable tasks are spread over the threads, computed now
  // and stored in the phi pass
  constexpr int PH = (2 * TT * NV + NT - 1) / NT;
  T phalo[PH];
  int phalo_at[PH];   // offset in sX (xlo: [0, NV NT), xhi: [NV NT, 2 NV NT)); -1: none
#pragma unroll
  for (int m = 0; m < PH; ++m) {
    const int t = tid + m * NT;
    phalo[m] = zero;
    phalo_at[m] = -1;
    if (t < 2 * TT * NV) {
      const int v = t / (2 * TT), h = t % (2 * TT);
      const int r = h % TT, f0 = r * (TP + 3);
      T a, b;
      if (h < TT) {
        slope_adj1(v, (r + 3) * HP + 2, 1, sFp, NFP, f0 + 1, f0, a, b);
        phalo[m] = b;
        phalo_at[m] = v * NT + r * TP;
      } else {
        slope_adj1(v, (r + 3) * HP + TP + 3, 1, sFp, NFP, f0 + TP + 2, f0 + TP + 1, a, b);
        phalo[m] = -a;
        phalo_at[m] = NV * NT + v * NT + r * TP + TP - 1;
      }
    }
  }
  // theta: own cell (jj, ii) is frame (jj + 3, ii + 3); its upper face is
  // theta face row jj + 2, its lower face row jj + 1
  {
    T dir[NV], ab[NV], bb[NV];
    slope_adj((jj + 3) * HP + ii + 3, HP, sFt, NFT, (jj + 2) * TP + ii, (jj + 1) * TP + ii, dir, ab, bb);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      acc[v] += dir[v];
      if (jj + 1 < TT) xlo[v * NT + tid + TP] = bb[v];
      if (jj >= 1) xhi[v * NT + tid - TP] = -ab[v];
    }
    // halo rows j0 - 1 (frame row 2, between theta face rows 0 and 1) and
    // j0 + TT (frame row TT + 3, between face rows TT + 1 and TT + 2) feed
    // rows 0 and TT - 1; their 2 TP x NV one-variable tasks are spread over
    // all threads
    for (int t = tid; t < 2 * TP * NV; t += NT) {
      const int v = t / (2 * TP), h = t % (2 * TP);
      const int c = h % TP;
      T a, b;
      if (h < TP) {
        slope_adj1(v, 2 * HP + c + 3, HP, sFt, NFT, TP + c, c, a, b);
        xlo[v * NT + c] = b;
      } else {
        slope_adj1(v, (TT + 3) * HP + c + 3, HP, sFt, NFT, (TT + 2) * TP + c, (TT + 1) * TP + c, a, b);
        xhi[v * NT + (TT - 1) * TP + c] = -a;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] += xlo[v * NT + tid] + xhi[v * NT + tid];
  __syncthreads();
  // phi: own cell's upper face is phi face col ii + 2 of row jj, lower ii + 1
  {
    T dir[NV], ab[NV], bb[NV];
    const int fb0 = jj * (TP + 3);
    slope_adj((jj + 3) * HP + ii + 3, 1, sFp, NFP, fb0 + ii + 2, fb0 + ii + 1, dir, ab, bb);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      acc[v] += dir[v];
      if (ii + 1 < TP) xlo[v * NT + tid + 1] = bb[v];
      if (ii >= 1) xhi[v * NT + tid - 1] = -ab[v];
    }
#pragma unroll
    for (int m = 0; m < PH; ++m)
      if (phalo_at[m] >= 0) sX[phalo_at[m]] = phalo[m];
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] += xlo[v * NT + tid] + xhi[v * NT + tid];

  // ---- the r part, the recovery adjoint (from the cell's primitives) and
  // the sources
  if (!own) return;
  T w[NV], ub[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    w[v] = sW[v * HC + (jj + 3) * HP + ii + 3];
    acc[v] += wr[v];
  }
  recover_adjoint_w(w, ph, acc, ub);
  const T gk = -g.grav[k];
  const T gx = gk * g.rhat[colo], gy = gk * g.rhat[cs + colo], gz = gk * g.rhat[2 * cs + colo];
  ub[0] += rsrc[0] * gx + rsrc[1] * gy + rsrc[2] * gz;   // S_m = rho g
  ub[1] += rsrc[3] * gx;                                 // S_E = m . g
  ub[2] += rsrc[3] * gy;
  ub[3] += rsrc[3] * gz;
  ub[8] -= ph.psi_damp * rsrc[4];                        // S_psi = -alpha psi
#pragma unroll
  for (int v = 0; v < NV; ++v) Ub[v * N + cell] = ub[v];
}

}  // namespace crn
