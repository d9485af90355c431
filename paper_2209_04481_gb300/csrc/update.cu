// update.cu -- explicit pseudo-time update of the FP64 master state and the
// res(a) convergence monitor of arXiv 2209.04481 Sect. 2.1.
//
// U^{t+1} = U^t + dt R(U^t), dt = cfl * dtmin, in FP64 on the master state.
// The monitor needs a^{t+1} - a^t for the nine primitives; it is formed from
// the increment dU = dt R without cancellation,
//   d rho = dU_rho,      dV = (dm - V^t d rho) / rho^{t+1},      dB = dU_B,
//   d(B^2/2) = B^t.dB + |dB|^2/2,
//   d(rho V^2/2) = (m^t.dm + |dm|^2/2 - rho^t |V^t|^2 d rho / 2) / rho^{t+1},
//   dp = (gamma - 1) (dE - d(rho V^2/2) - d(B^2/2)),   d psi = dU_psi,
// in the grid's precision, squared and summed per thread (compensated in
// FP32), then across threads and CTAs in FP64.
//
// FP32-bulk grids: the FP64 pipe executes only the nine master-state FMAs
// per cell.  Widening R and narrowing the new shadow go through the integer
// pipe (fp_bits.cuh), and the compensated FP32 sums are combined across the
// block in FP32 pairs before the one conversion to FP64 per block.
#include "corona_internal.h"
#include "fp_bits.cuh"
#include "residual.cuh"

namespace crn {

template <class TM>
__device__ __forceinline__ void monitor_increments(const TM (&u0)[NV], const TM (&du)[NV], TM gm1,
                                                   TM (&dw)[NV]) {
  const TM r0 = u0[0], dr = du[0];
  const TM r1 = r0 + dr;
  const TM ir0 = frcp(r0), ir1 = frcp(r1);
  const TM vx = u0[1] * ir0, vy = u0[2] * ir0, vz = u0[3] * ir0;
  dw[0] = dr;
  dw[1] = (du[1] - vx * dr) * ir1;
  dw[2] = (du[2] - vy * dr) * ir1;
  dw[3] = (du[3] - vz * dr) * ir1;
  dw[4] = du[4]; dw[5] = du[5]; dw[6] = du[6];
  const TM db = u0[4] * du[4] + u0[5] * du[5] + u0[6] * du[6]
                + (TM)0.5 * (du[4] * du[4] + du[5] * du[5] + du[6] * du[6]);
  const TM dk = (u0[1] * du[1] + u0[2] * du[2] + u0[3] * du[3]
                 + (TM)0.5 * (du[1] * du[1] + du[2] * du[2] + du[3] * du[3])
                 - (TM)0.5 * (u0[1] * vx + u0[2] * vy + u0[3] * vz) * dr) * ir1;
  dw[7] = gm1 * (du[7] - dk - db);
  dw[8] = du[8];
}

__device__ __forceinline__ double widen(float x) { return widen_f32(x); }
__device__ __forceinline__ double widen(double x) { return x; }

// (s, c) += (s2, c2) for compensated sums whose value is s - c: the sum of
// the leading parts is split exactly into t + err (Knuth's TwoSum), and err
// moves into the correction.
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
  const float t = s + s2;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (s2 - bp);
  s = t;
  c = (c + c2) - err;
}

// Block sum of the per-thread compensated FP32 sums (256 threads): FP32
// pairs across each warp by shuffles, then across the eight warps by warp 0;
// tot[] of thread 0 receives the block's totals, every other thread's tot[]
// is zero (the form reduce_and_finalize_at<256, true> takes, which adds the
// warps' lane-0 values).  `scratch` holds at least 8 * 2 * NV floats.
__device__ __forceinline__ void block_sum_pairs(Acc<float>& acc, double (&tot)[NV], double* scratch) {
  float* sp = reinterpret_cast<float*>(scratch);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float s2 = __shfl_xor_sync(0xffffffffu, acc.s[v], off);
      const float c2 = __shfl_xor_sync(0xffffffffu, acc.c[v], off);
      pair_add(acc.s[v], acc.c[v], s2, c2);
    }
  }
  __syncthreads();  // scratch may still be read by an earlier use
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sp[(warp * NV + v) * 2] = acc.s[v];
      sp[(warp * NV + v) * 2 + 1] = acc.c[v];
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = 0.0;
  if (warp == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float s = 0.f, c = 0.f;
      if (lane < 8) {
        s = sp[(lane * NV + v) * 2];
        c = sp[(lane * NV + v) * 2 + 1];
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, off);
        pair_add(s, c, s2, c2);
      }
      if (lane == 0) tot[v] = (double)s - (double)c;
    }
  }
}

// U^t, R and the state the monitor differences against (the FP32 shadow
// when there is one) of cell c
template <class TR>
__device__ __forceinline__ void load_cell(int64_t N, int64_t c, const double* __restrict__ U,
                                          const TR* __restrict__ R, const float* shadow_old,
                                          double (&uo)[NV], TR (&r)[NV], TR (&u0)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    uo[v] = U[v * N + c];
    r[v] = R[v * N + c];
  }
  if (shadow_old) {
#pragma unroll
    for (int v = 0; v < NV; ++v) u0[v] = (TR)shadow_old[v * N + c];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) u0[v] = (TR)uo[v];
  }
}

// TR: element type of R (double on FP64 grids, float on FP32_BULK grids);
// the monitor arithmetic runs in the same type.
// block `bid` of `nblocks` blocks covering the N cells of one grid
template <class TR>
__device__ __forceinline__ void update_block(int64_t N, double* __restrict__ U, const TR* __restrict__ R,
                                             const float* shadow_old, float* shadow_new,
                                             const double* __restrict__ dtmin, double cfl, TR gm1,
                                             const Reduce& red, int bid, int nblocks, double* scratch) {
  const double dt = cfl * dtmin[0];
  const TR dtr = (TR)dt;
  Acc<TR> acc;
  acc.init();
  // one cell: master-state update, new shadow, monitor increments
  auto step = [&](int64_t c, const double (&uo)[NV], const TR (&r)[NV], const TR (&u0)[NV]) {
    TR du[NV], dw[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double un = fma(dt, widen(r[v]), uo[v]);
      U[v * N + c] = un;
      if (shadow_new) shadow_new[v * N + c] = narrow_f64(un);
      du[v] = dtr * r[v];
    }
    monitor_increments(u0, du, gm1, dw);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc.add(v, dw[v]);
  };
  // all 27 loads of a cell are issued before its first store: the old and
  // the new shadow are one buffer, so interleaving them would serialise nine
  // memory round trips per cell
  const int64_t stride = (int64_t)nblocks * blockDim.x;
  for (int64_t c = (int64_t)bid * blockDim.x + threadIdx.x; c < N; c += stride) {
    double uo[NV];
    TR r[NV], u0[NV];
    load_cell(N, c, U, R, shadow_old, uo, r, u0);
    step(c, uo, r, u0);
  }
  double tot[NV];
  if constexpr (std::is_same<TR, float>::value) {
    block_sum_pairs(acc, tot, scratch);
    reduce_and_finalize_at<256, true>(tot, INFINITY, red, scratch, bid, nblocks);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) tot[v] = acc.total(v);
    reduce_and_finalize_at<256>(tot, INFINITY, red, scratch, bid, nblocks);
  }
}

template <class TR>
__global__ void __launch_bounds__(256)
update_kernel(int64_t N, double* __restrict__ U, const TR* __restrict__ R,
              const float* shadow_old, float* shadow_new,
              const double* __restrict__ dtmin, double cfl, TR gm1, Reduce red) {
  __shared__ double scratch[8 * RED_STRIDE];
  update_block<TR>(N, U, R, shadow_old, shadow_new, dtmin, cfl, gm1, red, blockIdx.x, gridDim.x, scratch);
}

// ensemble: one block per (member, block) item, members numbered in order
struct EnsUpdate {
  int64_t N;
  double* U;
  const void* R;       // the member's residual buffer (FP32 or FP64)
  float* shadow;       // FP32 shadow (FP32-bulk members), else null
  const double* dtmin;
  double gm1;
  Reduce red;
  int item0, nitems;
};

template <class TR>
__global__ void __launch_bounds__(256)
ensemble_update_kernel(const EnsUpdate* __restrict__ mem, int nmem, double cfl) {
  __shared__ double scratch[8 * RED_STRIDE];
  const int item = blockIdx.x;
  int m = 0;
  while (m + 1 < nmem && mem[m + 1].item0 <= item) ++m;
  const EnsUpdate& M = mem[m];
  update_block<TR>(M.N, M.U, static_cast<const TR*>(M.R), M.shadow, M.shadow, M.dtmin, cfl, (TR)M.gm1,
                   M.red, item - M.item0, M.nitems, scratch);
}

size_t ens_update_bytes() { return sizeof(EnsUpdate); }

void ens_update_fill(crn_grid* g, double* U64, int item0, int nitems, double* log_out, void* dst) {
  EnsUpdate* m = static_cast<EnsUpdate*>(dst);
  m->N = g->shape.ncell;
  m->U = U64;
  m->R = g->rbuf;
  m->shadow = g->d.precision == CRN_FP64 ? nullptr : g->shadow;
  m->dtmin = g->stats + 9;
  m->gm1 = g->d.gamma - 1.0;
  Reduce& red = m->red;
  red.partials = g->partials;
  red.counter = g->counter;
  red.norms_out = nullptr;
  red.dt_out = nullptr;
  red.norms_user = nullptr;
  red.dt_user = nullptr;
  red.err_flags = g->err_flags;
  red.err_cell = g->err_cell;
  red.log_out = log_out ? log_out : g->stats + 10;
  m->item0 = item0;
  m->nitems = nitems;
}

cudaError_t launch_ensemble_update(const void* dev, int nmem, int nitems, double cfl, bool fp32,
                                   cudaStream_t st) {
  const EnsUpdate* m = static_cast<const EnsUpdate*>(dev);
  if (fp32)
    ensemble_update_kernel<float><<<nitems, 256, 0, st>>>(m, nmem, cfl);
  else
    ensemble_update_kernel<double><<<nitems, 256, 0, st>>>(m, nmem, cfl);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
shadow_kernel(int64_t n, const double* __restrict__ U, float* __restrict__ S) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    S[q] = (float)U[q];
}

// Resident 256-thread blocks per SM of the update kernel (register bound).
int update_blocks_per_sm(bool fp32) {
  int n = 0;
  const cudaError_t e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, update_kernel<float>, 256, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, update_kernel<double>, 256, 0);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    n = 2;
  }
  return n < 1 ? 1 : n;
}

// Blocks of the update: one resident wave, grid-stride.  The closing
// last-CTA reduction costs every block a partial, an arrival atomic on one
// counter, and a row the last CTA reads back; on 128 x 64 x 128 each block
// beyond the first wave cost about 17 ns, and a second wave gave no overlap
// that paid for it.
unsigned update_blocks(const crn_grid* g) {
  int64_t nb = (g->shape.ncell + 255) / 256;
  const int64_t cap = (int64_t)g->cfg.update_per_sm * g->cfg.num_sms;
  if (nb > cap) nb = cap;
  if (nb > (int64_t)g->max_blocks) nb = (int64_t)g->max_blocks;
  return (unsigned)(nb < 1 ? 1 : nb);
}

cudaError_t launch_update(crn_grid* g, double* U64, double cfl, double* res_out,
                          cudaStream_t st, int* nlaunch) {
  Reduce red;
  red.partials = g->partials;
  red.counter = g->counter;
  red.norms_out = nullptr;
  red.dt_out = nullptr;
  red.norms_user = nullptr;
  red.dt_user = nullptr;
  red.err_flags = g->err_flags;
  red.err_cell = g->err_cell;
  // the monitor always writes somewhere: the caller's row or the grid's stats
  red.log_out = res_out ? res_out : g->stats + 10;
  const unsigned nb = update_blocks(g);
  *nlaunch = 1;
  if (g->d.precision == CRN_FP64) {
    update_kernel<double><<<nb, 256, 0, st>>>(g->shape.ncell, U64, (const double*)g->rbuf,
                                              nullptr, nullptr, g->stats + 9, cfl,
                                              g->ph64.gm1, red);
  } else {
    // the residual of this step was evaluated on the current shadow, which
    // therefore still holds U^t; the new shadow is written in place
    update_kernel<float><<<nb, 256, 0, st>>>(g->shape.ncell, U64, (const float*)g->rbuf,
                                             g->shadow, g->shadow, g->stats + 9, cfl,
                                             g->ph32.gm1, red);
  }
  return cudaGetLastError();
}

cudaError_t launch_shadow(crn_grid* g, const double* U64, cudaStream_t st, int* nlaunch) {
  const int64_t n = 9 * g->shape.ncell;
  int64_t nb = (n + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  shadow_kernel<<<(unsigned)nb, 256, 0, st>>>(n, U64, g->shadow);
  *nlaunch = 1;
  return cudaGetLastError();
}

}  // namespace crn
