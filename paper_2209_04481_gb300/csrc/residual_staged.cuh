// residual_staged.cuh -- the FP32-bulk production residual kernel for sm_103a.
//
// Same operator as residual.cuh (arXiv 2209.04481: Sect. 2.1 second-order FV
// with hyperbolic divergence cleaning, Sect. 2.2 equations and gravity
// sources, Sect. 3.2 inner boundary, Sect. 4.1 / Table 2 outer boundary),
// organised for GB300's issue rate:
//
//  * Staging.  A CTA owns a TT x TP block of (theta, phi) columns and marches
//    outwards in r.  The raw state of each plane's own block (TT x TP cells x
//    9 variables) arrives by one TMA tensor copy (cp.async.bulk.tensor, 4D map
//    over [var][r][theta][phi]) completing on an mbarrier; the 4 TP + 4 TT halo
//    cells the stencils need (two rows above and below, two columns either
//    side; across the poles and the periodic seam) arrive by 4-byte cp.async
//    copies of the threads that recover them.  Two raw stages are in flight
//    ahead of the plane being recovered, so no thread holds prefetched data in
//    registers.
//  * One recovery per cell and plane into a 3-plane ring of primitives.
//  * Faces computed once each, with their reconstructed states built on the
//    fly from the 4-cell stencil in shared memory (no stored face values).
//  * Every thread evaluates its cell's lower theta and phi faces; the first
//    TT + TP threads also take one face on the far side of the block (row TT
//    of theta faces, column TP of phi faces); after the barrier each thread
//    evaluates its upper r face and gathers.  Two barriers per plane.
//  * Gather, gravity, norms and the step bound as in the tiled kernel; the
//    cross-warp and cross-CTA reduction in FP64 in a fixed order.
//
// Requirements (checked on the host): n_theta % TT == 0, n_phi % TP == 0 (no
// ragged blocks: every own cell is inside the shell, so the TMA box never
// leaves it), FP32 state 16-byte aligned.
#pragma once

#include <cuda.h>

#include "residual.cuh"

namespace crn {

// ---------------------------------------------------------------------------
// asynchronous copies and mbarriers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make barrier initialisation and earlier generic-proxy accesses of shared
// memory visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Bounded wait for the phase of `parity` to complete: gives up and returns
// false once `limit` SM clock cycles have passed (the caller reports
// CRN_E_TIMEOUT instead of spinning on a copy that never lands).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// 4D tiled TMA load of box {x, y, z, w} (innermost first) into shared memory,
// completing `bytes` of the mbarrier's expected transaction count
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Reconstructed states of the face between s1 and s2 of a unit-spaced
// stencil s0 s1 | s2 s3: wl = upper value of s1's cell, wr = lower value of
// s2's cell (the same operations, in the same order, as the tiled kernel's
// stored face values).
template <int LIM>
__device__ __forceinline__ void face_states1(float s0, float s1, float s2, float s3, float eps, float& wl,
                                             float& wr) {
  const float sl = limited_slope<LIM>(s1 - s0, s2 - s1, eps);
  const float sr = limited_slope<LIM>(s2 - s1, s3 - s2, eps);
  wl = fmaf(0.5f, sl, s1);
  wr = fmaf(-0.5f, sr, s2);
}

// ---------------------------------------------------------------------------
// shapes and shared-memory layout
// ---------------------------------------------------------------------------
template <int TT, int TP>
struct StagedDims {
  static constexpr int NT = TT * TP;              // threads, one cell each
  static constexpr int NTH = NT;
  static constexpr int HT = TT + 4, HP = TP + 4;  // halo'd plane (2 cells each side)
  static constexpr int HC = HT * HP;
  static constexpr int NH = 4 * TP + 4 * TT;      // halo cells the stencils read
  static constexpr int NH_OWN = NH;              // recovered by threads 0 .. NH - 1
  static constexpr int NTV = (TT + 1) * TP;       // theta faces (rows 0..TT)
  static constexpr int NPV = TT * (TP + 1);       // phi faces (cols 0..TP)
  static constexpr int NF = NV + 1;               // 9 fluxes + lambda |S|
  static constexpr int NEDGE = TP + TT;           // far-side faces per plane (threads 0 .. NEDGE - 1)
  static constexpr int NGEO = 3 * NTV + 2 * (TP + 1) + 6 * NT + (TT + 1) + 2 * TT;
  static constexpr size_t RAW = ((size_t)NV * NT * 4 + 1023) / 1024 * 1024;  // one TMA stage
  static constexpr size_t RAWH = (size_t)NV * NH * 4;                        // one halo stage
  static constexpr size_t OFF_HALO = 2 * RAW;
  static constexpr size_t OFF_RING = OFF_HALO + 2 * RAWH;
  static constexpr size_t OFF_FLUX = OFF_RING + (size_t)3 * NV * HC * 4;
  static constexpr size_t OFF_GEO = OFF_FLUX + (size_t)NF * (NTV + NPV) * 4;
  static constexpr size_t OFF_BAR = (OFF_GEO + (size_t)NGEO * 4 + 15) / 16 * 16;
  static constexpr size_t BYTES = OFF_BAR + 16 + 1024;  // + slack to align the base to 1024 B
  static_assert(NT % 32 == 0, "threads fill whole warps");
  static_assert(NH <= NT && NEDGE <= NT, "halo and far-side face assignment");
  static_assert(TT <= 32 && TP <= 256 && NV <= 256, "TMA box limits");
  // halo cell h in [0, NH) -> halo'd (row, col)
  __device__ static void halo_rc(int h, int& row, int& col) {
    if (h < 2 * TP) { row = h / TP; col = h % TP + 2; }
    else if (h < 4 * TP) { h -= 2 * TP; row = TT + 2 + h / TP; col = h % TP + 2; }
    else { h -= 4 * TP; row = 2 + h / 4; const int c = h % 4; col = c < 2 ? c : TP + c; }
  }
};

// per-CTA state that persists across the work items of a persistent launch
struct StagedCta {
  uint32_t phase;  // parity bit of each TMA stage's mbarrier
};

// SM clock cycles a thread waits for a TMA copy before reporting a timeout
// (about one second at GB300's 2 GHz; a plane's copy takes microseconds)
constexpr long long kTmaWaitCycles = 2000000000ll;

// One work item: tile `tile` (row-major over the (theta, phi) blocks) and
// radial chunk `chunk` of one grid; `bid` / `nblocks` number the items of that
// grid for its cross-CTA reduction.  All threads of the CTA call it.
template <int LIM, int TT, int TP>
__device__ __forceinline__ void staged_item(const Shape& sh, const Geo<float>& g, const Phys<float>& ph,
                                            const double* __restrict__ Br, const float* __restrict__ U,
                                            float* __restrict__ R, const Reduce& red, const CUtensorMap* tmap,
                                            int kchunk, int tile, int chunk, int bid, int nblocks,
                                            unsigned char* smem, StagedCta& cta) {
  using D = StagedDims<TT, TP>;
  constexpr int NT = D::NT, HP = D::HP, HC = D::HC, NTV = D::NTV, NPV = D::NPV, NF = D::NF, NH = D::NH;
  float* const raw = reinterpret_cast<float*>(smem);                   // [2][NV][TT][TP] (stride RAW)
  float* const rawh = reinterpret_cast<float*>(smem + D::OFF_HALO);    // [2][NV][NH]
  float* const ring = reinterpret_cast<float*>(smem + D::OFF_RING);    // [3][NV][HC]
  float* const ft = reinterpret_cast<float*>(smem + D::OFF_FLUX);      // [NF][NTV]  theta-face flux x |S|
  float* const fpf = ft + NF * NTV;                                    // [NF][NPV]  phi-face flux x |S|
  float* const s_nth = reinterpret_cast<float*>(smem + D::OFF_GEO);   // [3][NTV]
  float* const s_nph = s_nth + 3 * NTV;                                // [2][TP + 1]
  float* const s_nr = s_nph + 2 * (TP + 1);                            // [3][NT]
  float* const s_rh = s_nr + 3 * NT;                                   // [3][NT]
  float* const s_at = s_rh + 3 * NT;                                   // [TT + 1]
  float* const s_ar = s_at + (TT + 1);                                 // [TT]
  float* const s_av = s_ar + TT;                                       // [TT]
  uint64_t* const bars = reinterpret_cast<uint64_t*>(smem + D::OFF_BAR);

  const int nr = sh.nr, nt = sh.nt, np = sh.np;
  const int64_t N = sh.ncell, cs = (int64_t)nt * np;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ntp = np / TP;
  const int j0 = (tile / ntp) * TT, i0 = (tile % ntp) * TP;
  const int k0 = chunk * kchunk;
  const int k1 = min(nr, k0 + kchunk);
  const int plast = min(k1 + 1, nr - 1);  // last plane whose raw state is loaded
  const int jj = tid / TP, ii = tid % TP;
  const int hown = (jj + 2) * HP + (ii + 2);
  const int64_t ocol = (int64_t)(j0 + jj) * np + (i0 + ii);
  const float eps = ph.eps;

  // halo cell of this thread (threads 0 .. NH - 1): its position in the
  // halo'd plane and its (across-pole / periodic) column in the shell
  const bool halo = tid < NH;
  int hpos = 0, hcol = 0;
  if (halo) {
    int row, col;
    D::halo_rc(tid, row, col);
    int jh = j0 - 2 + row, ih = i0 - 2 + col;
    map_column(jh, ih, nt, np);
    hpos = row * HP + col;
    hcol = jh * np + ih;
  }

  // per-CTA geometry
  {
    const int64_t ts = (int64_t)(nt + 1) * np;
    for (int q = tid; q < NTV; q += D::NTH) {
      const int f = q / TP, col = q % TP;
      const int64_t fc = (int64_t)min(j0 + f, nt) * np + (i0 + col);
      s_nth[q] = g.nth[fc];
      s_nth[NTV + q] = g.nth[ts + fc];
      s_nth[2 * NTV + q] = g.nth[2 * ts + fc];
    }
    for (int q = tid; q <= TP; q += D::NTH) {
      int ic = i0 + q;
      ic = ic >= np ? ic - np : ic;
      s_nph[q] = g.nph[ic];
      s_nph[TP + 1 + q] = g.nph[np + ic];
    }
    {
      s_nr[tid] = g.nr[ocol];
      s_nr[NT + tid] = g.nr[cs + ocol];
      s_nr[2 * NT + tid] = g.nr[2 * cs + ocol];
      s_rh[tid] = g.rhat[ocol];
      s_rh[NT + tid] = g.rhat[cs + ocol];
      s_rh[2 * NT + tid] = g.rhat[2 * cs + ocol];
    }
    if (tid <= TT) s_at[tid] = g.at[min(j0 + tid, nt)];
    if (tid < TT) {
      s_ar[tid] = g.ar[j0 + tid];
      s_av[tid] = g.av[j0 + tid];
    }
  }

  auto slot = [&](int p) -> float* { return ring + (p % 3) * (NV * HC); };

  // request the raw state of plane p into stage p & 1 (TMA for the own block,
  // cp.async for the halo); one cp.async group per plane, empty past plast
  auto issue = [&](int p) {
    if (p <= plast) {
      const int b = p & 1;
      if (tid == 0) {  // the TMA issuer
        fence_proxy_async();
        mbar_expect_tx(&bars[b], (uint32_t)(NV * NT * 4));
        tma_load_4d(smem + b * D::RAW, tmap, i0, j0, p, 0, &bars[b]);
      }
      if (p < k1 && halo) {  // planes past the chunk: own column only
        const float* src = U + (int64_t)p * cs + hcol;
        float* dst = rawh + b * (NV * NH) + tid;
#pragma unroll
        for (int v = 0; v < NV; ++v) cp_async4(dst + v * NH, src + v * N);
      }
    }
    cp_async_commit();
  };

  // recover plane p into the ring (p <= plast), or form the outer ghost plane
  // of the own column (p == nr); returns false if the TMA wait timed out
  auto consume = [&](int p) -> bool {
    if (p > nr) return true;
    float* dst = slot(p);
    if (p == nr) {  // outer ghost [Sect. 4.1 / Table 2]: own column only
      const float* src = slot(nr - 1);
      float wi[NV], wg[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wi[v] = src[v * HC + hown];
      outer_ghost(wi, s_rh[tid], s_rh[NT + tid], s_rh[2 * NT + tid], ph, wg);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + hown] = wg[v];
      return true;
    }
    const int b = p & 1;
    bool ok = true;
    cp_async_wait<1>();
    ok = mbar_wait(&bars[b], (cta.phase >> b) & 1u, kTmaWaitCycles);
    cta.phase ^= 1u << b;
    if (ok) {
      const float* src = raw + b * (D::RAW / 4) + tid;
      float u[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = src[v * NT];
      recover(u, ph, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + hown] = w[v];
    }
    if (p < k1 && halo) {
      const float* src = rawh + b * (NV * NH) + tid;
      float u[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = src[v * NH];
      recover(u, ph, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * HC + hpos] = w[v];
    }
    return ok;
  };

  // own-column r values of plane p: lower (lo) and upper (up) face values
  // from planes p - 1, p, p + 1 (distance-weighted slopes)
  auto r_values = [&](int p, const float (&wm)[NV], const float (&w0)[NV], const float (&wp)[NV], float (&lo)[NV],
                      float (&up)[NV]) {
    const float im = g.inv_dm[p], ip = g.inv_dp[p], hm = g.hm[p], hp = g.hp[p];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float s = limited_slope<LIM>((w0[v] - wm[v]) * im, (wp[v] - w0[v]) * ip, eps);
      lo[v] = fmaf(-s, hm, w0[v]);
      up[v] = fmaf(s, hp, w0[v]);
    }
  };

  bool bad = false;
  // ---------------- preamble: planes k0, k0 + 1 in the ring; r face k0 - 1/2
  issue(k0);
  issue(k0 + 1);
  float rL[NV];   // left state of r face k + 1/2 (upper r value of plane k)
  float frl[NF];  // flux x area of r face k - 1/2, lambda x area last
  float um1[NV], um2[NV];
  {  // own column of planes k0 - 1 and k0 - 2 (plain loads)
    if (k0 >= 1) load_raw(U + (int64_t)(k0 - 1) * cs, N, ocol, um1);
    if (k0 >= 2) load_raw(U + (int64_t)(k0 - 2) * cs, N, ocol, um2);
  }
  bad |= !consume(k0);
  bad = __syncthreads_or(bad);
  if (!bad) {
    issue(k0 + 2);
    bad |= !consume(k0 + 1);
  }
  bad = __syncthreads_or(bad);
  if (!bad) issue(k0 + 3);
  if (!bad) {
    float w0[NV], w1[NV], wm1[NV], wm2[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      w0[v] = slot(k0)[v * HC + hown];
      w1[v] = slot(k0 + 1)[v * HC + hown];
    }
    const double ex = (double)g.rhat[ocol], ey = (double)g.rhat[cs + ocol], ez = (double)g.rhat[2 * cs + ocol];
    if (k0 >= 1) recover(um1, ph, wm1);
    else inner_ghost_at(w0, Br, ocol, cs, ex, ey, ez, ph, wm1);  // [Sect. 3.2]
    if (k0 >= 2) recover(um2, ph, wm2);
    else if (k0 == 1) {
      float wz[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wz[v] = wm1[v];  // plane 0
      inner_ghost_at(wz, Br, ocol, cs, ex, ey, ez, ph, wm2);
    }
    float up0[NV], lo0[NV];
    r_values(k0, wm1, w0, w1, lo0, up0);
    float wl[NV], wr[NV];
    if (k0 == 0) {  // inner boundary face: first order, ghost | interior
#pragma unroll
      for (int v = 0; v < NV; ++v) { wl[v] = wm1[v]; wr[v] = w0[v]; }
    } else {
      float lo[NV];
      r_values(k0 - 1, wm2, wm1, w0, lo, wl);
#pragma unroll
      for (int v = 0; v < NV; ++v) wr[v] = lo0[v];
    }
    float f[NV], la;
    rusanov(wl, wr, s_nr[tid], s_nr[NT + tid], s_nr[2 * NT + tid], g.ra[k0] * s_ar[jj], ph, f, la);
#pragma unroll
    for (int v = 0; v < NV; ++v) frl[v] = f[v];
    frl[NV] = la;
#pragma unroll
    for (int v = 0; v < NV; ++v) rL[v] = up0[v];
  }

  float sq[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sq[v] = 0.f;
  float dtm = INFINITY;

  for (int k = k0; k < k1 && !bad; ++k) {
    // ---- A: plane k + 2 enters the ring; its stage is then refilled with plane k + 4
    bad |= !consume(k + 2);
    bad = __syncthreads_or(bad);
    if (bad) break;
    issue(k + 4);
    // ---- B: every theta and phi face of plane k once (each thread its cell's
    //         lower faces; threads 0 .. TP + TT - 1 also theta row TT or phi
    //         column TP)
    const float* P = slot(k);
    const float rbk = g.rb[k];
    const int nface = tid < D::NEDGE ? 3 : 2;
#pragma unroll 1
    for (int it = 0; it < nface; ++it) {
      // face kind 0: theta, 1: phi; stencil centre (upper cell) and stride in the ring
      bool theta, live = true;
      int base, q, f;
      if (it < 2) {
        theta = it == 0;
        base = hown;
        q = theta ? jj * TP + ii : jj * (TP + 1) + ii;
        f = ii;
        live = !theta || j0 + jj > 0;  // the north pole face has zero area
      } else {
        const int e = tid;
        theta = e < TP;
        if (theta) {  // theta face row TT, column e (the south pole face if j0 + TT == nt)
          base = (TT + 2) * HP + (e + 2);
          q = TT * TP + e;
          live = j0 + TT < nt;
        } else {      // phi face column TP, row e - TP
          base = (e - TP + 2) * HP + (TP + 2);
          q = (e - TP) * (TP + 1) + TP;
        }
        f = TP;
      }
      const int stride = theta ? HP : 1;
      float wl[NV], wr[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* c = P + v * HC + base;
        face_states1<LIM>(c[-2 * stride], c[-stride], c[0], c[stride], eps, wl[v], wr[v]);
      }
      float nx, ny, nz, area;
      if (theta) {
        nx = s_nth[q];
        ny = s_nth[NTV + q];
        nz = s_nth[2 * NTV + q];
        area = rbk * s_at[q / TP];
      } else {
        nx = s_nph[f];
        ny = s_nph[TP + 1 + f];
        nz = 0.f;
        area = rbk * g.dtheta;
      }
      float fl[NV], la;
      rusanov(wl, wr, nx, ny, nz, area, ph, fl, la);
      float* out = theta ? ft : fpf;
      const int ns = theta ? NTV : NPV;
#pragma unroll
      for (int v = 0; v < NV; ++v) out[v * ns + q] = live ? fl[v] : 0.f;
      out[NV * ns + q] = live ? la : 0.f;
    }
    __syncthreads();
    // ---- C: the own column's upper r face k + 1/2, then the gather of the six
    //         faces of cell (k, j0 + jj, i0 + ii)
    {
      float fru[NF];
      {
        float wl[NV], wr[NV];
        if (k + 1 < nr) {
          float w0[NV], w1[NV], w2[NV], rLn[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            w0[v] = P[v * HC + hown];
            w1[v] = slot(k + 1)[v * HC + hown];
            w2[v] = slot(k + 2)[v * HC + hown];
          }
          r_values(k + 1, w0, w1, w2, wr, rLn);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            wl[v] = rL[v];
            rL[v] = rLn[v];
          }
        } else {  // outer boundary face: first order, interior | ghost
          const float* pg = slot(nr);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            wl[v] = P[v * HC + hown];
            wr[v] = pg[v * HC + hown];
          }
        }
        float fl[NV], la;
        rusanov(wl, wr, s_nr[tid], s_nr[NT + tid], s_nr[2 * NT + tid], g.ra[k + 1] * s_ar[jj], ph, fl, la);
#pragma unroll
        for (int v = 0; v < NV; ++v) fru[v] = fl[v];
        fru[NV] = la;
      }
      const int tl = jj * TP + ii, tu = tl + TP;
      const int pl = jj * (TP + 1) + ii, pu = pl + 1;
      float r[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        r[v] = (frl[v] - fru[v]) + (ft[v * NTV + tl] - ft[v * NTV + tu]) + (fpf[v * NPV + pl] - fpf[v * NPV + pu]);
      const float lam = (frl[NV] + fru[NV]) + (ft[NV * NTV + tl] + ft[NV * NTV + tu]) +
                        (fpf[NV * NPV + pl] + fpf[NV * NPV + pu]);
      const float vol = g.rv[k] * s_av[jj];
      const float ivol = 1.f / vol;
#pragma unroll
      for (int v = 0; v < NV; ++v) r[v] *= ivol;
      const float rho = P[hown], vx = P[HC + hown], vy = P[2 * HC + hown], vz = P[3 * HC + hown];
      const float pr = P[7 * HC + hown], psi = P[8 * HC + hown];
      const float gk = -g.grav[k];  // gravity [Sect. 2.2]: rho g, rho g.V
      const float gx = gk * s_rh[tid], gy = gk * s_rh[NT + tid], gz = gk * s_rh[2 * NT + tid];
      r[1] += rho * gx;
      r[2] += rho * gy;
      r[3] += rho * gz;
      r[7] += rho * (vx * gx + vy * gy + vz * gz);
      r[8] -= ph.psi_damp * psi;
      const int64_t cell = (int64_t)k * cs + ocol;
      float chk = 0.f;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R[v * N + cell] = r[v];
        sq[v] = fmaf(r[v], r[v], sq[v]);
        chk = fmaf(r[v], r[v], chk);
      }
      const float dtc = vol / lam;
      dtm = dtc < dtm ? dtc : dtm;
      if (!(rho > 0.f) || !(pr > 0.f) || !(fabsf(chk) < INFINITY)) flag_bad(red, cell);
#pragma unroll
      for (int v = 0; v < NF; ++v) frl[v] = fru[v];
    }
  }
  if (bad) {
    // a TMA copy did not complete: report it, drain this thread's cp.async
    // copies and leave the item with empty partials (the cross-CTA reduction
    // still completes, so the arrival counter stays consistent)
    if (tid == 0) atomicOr(red.err_flags, 2u);
    cp_async_wait<0>();
#pragma unroll
    for (int v = 0; v < NV; ++v) sq[v] = 0.f;
    dtm = INFINITY;
  }
  // ---------------- reductions: warp tree in FP32, then FP64 across warps and CTAs
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sq[v] += __shfl_xor_sync(0xffffffffu, sq[v], off);
    const float o = __shfl_xor_sync(0xffffffffu, dtm, off);
    dtm = o < dtm ? o : dtm;
  }
  double tot[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = lane == 0 ? (double)sq[v] : 0.0;
  double* scratch = reinterpret_cast<double*>(ft);
  reduce_and_finalize_at<D::NTH, true>(tot, (double)dtm, red, scratch, bid, nblocks);
}

// the 1024-byte aligned base of the dynamic shared memory
__device__ __forceinline__ unsigned char* staged_smem_base(unsigned char* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  return reinterpret_cast<unsigned char*>((a + 1023) & ~static_cast<uintptr_t>(1023));
}

template <int TT, int TP>
__device__ __forceinline__ void staged_init(unsigned char* smem, StagedCta& cta) {
  using D = StagedDims<TT, TP>;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + D::OFF_BAR);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  cta.phase = 0u;
  __syncthreads();
}

// one grid: block (x, y) = (tile, radial chunk)
template <int LIM, int TT, int TP>
__global__ void __launch_bounds__(TT * TP, 2)
residual_staged(Shape sh, Geo<float> g, Phys<float> ph, const double* __restrict__ Br,
                const float* __restrict__ U, float* __restrict__ R, Reduce red, int kchunk,
                const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = staged_smem_base(smem_raw);
  StagedCta cta;
  staged_init<TT, TP>(smem, cta);
  staged_item<LIM, TT, TP>(sh, g, ph, Br, U, R, red, &tmap, kchunk, blockIdx.x, blockIdx.y,
                           blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y, smem, cta);
}

}  // namespace crn
