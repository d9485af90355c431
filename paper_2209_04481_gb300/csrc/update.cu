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
#include "corona_internal.h"
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
  for (int64_t c = (int64_t)bid * blockDim.x + threadIdx.x; c < N; c += (int64_t)nblocks * blockDim.x) {
    TR u0[NV], du[NV], dw[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double uo = U[v * N + c];
      const TR r = R[v * N + c];
      // the old shadow (if any) is read before the new one overwrites it
      u0[v] = shadow_old ? (TR)shadow_old[v * N + c] : (TR)uo;
      const double un = fma(dt, (double)r, uo);
      U[v * N + c] = un;
      if (shadow_new) shadow_new[v * N + c] = (float)un;
      du[v] = dtr * r;
    }
    monitor_increments(u0, du, gm1, dw);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc.add(v, dw[v]);
  }
  double tot[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = acc.total(v);
  reduce_and_finalize_at<256>(tot, INFINITY, red, scratch, bid, nblocks);
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

unsigned update_blocks(const crn_grid* g) {
  int64_t nb = (g->shape.ncell + 255) / 256;
  if (nb > (int64_t)g->max_blocks) nb = (int64_t)g->max_blocks;
  if (nb > 4 * 152 * 8) nb = 4 * 152 * 8;
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
