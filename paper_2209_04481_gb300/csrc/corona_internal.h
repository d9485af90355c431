// corona_internal.h -- host-side grid object and kernel launchers shared by
// the translation units of libcorona (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "../../include/corona.h"
#include "mhd_device.cuh"

namespace crn {

struct Reduce;
struct NkWork;                // Newton-Krylov workspace (nk.cu)
void nk_free(NkWork* w);
struct HostPipe;              // host-buffer staging (host_io.cu)
void host_pipe_free(HostPipe* p);

// device geometry of one precision (one allocation, carved into arrays)
template <class T>
struct GeoBuf {
  T* base = nullptr;
  Geo<T> geo{};
};

struct LaunchCfg {
  int kchunk_tiled = 16;  // radial planes per CTA of the tiled kernel
  int num_sms = 152;      // streaming multiprocessors of the grid's device
  int update_per_sm = 2;  // resident blocks per SM of the pseudo-time update
  bool staged = false;    // FP32 residuals use the TMA-staged kernel (on request)
  int kchunk_staged = 16; // radial planes per CTA of the staged kernel
};

}  // namespace crn

struct crn_grid {
  crn_grid_desc d;
  int device = 0;
  crn::Shape shape{};
  crn::Phys<double> ph64{};
  crn::Phys<float> ph32{};
  crn::GeoBuf<double> g64;
  crn::GeoBuf<float> g32;
  double* br = nullptr;            // [nt][np] prescribed B_r
  bool have_br = false;
  double* partials = nullptr;      // reduction partials [max_blocks][16]
  size_t max_blocks = 0;
  unsigned int* counter = nullptr; // CTA arrival counter
  double* stats = nullptr;         // [0..8] norms, [9] dtmin
  unsigned int* err_flags = nullptr;
  unsigned long long* err_cell = nullptr;
  void* rbuf = nullptr;            // residual scratch for pseudo-time stepping (9N of T)
  void* vjp_buf = nullptr;         // VJP face contributions (allocated by the first VJP call)
  float* shadow = nullptr;         // FP32 shadow of the master state (FP32_BULK)
  crn::NkWork* nk = nullptr;       // Newton-Krylov workspace (allocated by the first NK call)
  crn::HostPipe* pipe = nullptr;   // host-buffer staging (allocated by the first host batch)
  int64_t last_bad_cell = -1;
  int32_t last_launches = 0;
  int32_t last_kernel = -1;        // crn_kernel of the last residual launch
  crn::LaunchCfg cfg;
};

namespace crn {

// launchers (return cudaGetLastError() of the launch)
cudaError_t launch_residual_fp64(crn_grid* g, const double* U, double* R, double* norms_user,
                                 double* dt_user, cudaStream_t st, int* nlaunch);
cudaError_t launch_residual_fp32(crn_grid* g, const float* U, float* R, double* norms_user,
                                 double* dt_user, cudaStream_t st, int* nlaunch);
cudaError_t launch_update(crn_grid* g, double* U64, double cfl, double* res_out,
                          cudaStream_t st, int* nlaunch);
cudaError_t launch_shadow(crn_grid* g, const double* U64, cudaStream_t st, int* nlaunch);
cudaError_t launch_vjp_fp64(crn_grid* g, const double* U, const double* Rb, double* Ub, double* Brb,
                            cudaStream_t st, int* nlaunch);
cudaError_t launch_vjp_fp32(crn_grid* g, const float* U, const float* Rb, float* Ub, double* Brb,
                            cudaStream_t st, int* nlaunch);
size_t vjp_scratch_bytes(const crn_grid* g);
// ensemble records (EnsMember<T> of residual.cuh, opaque here) and launches
size_t ens_member_bytes_fp64();
size_t ens_member_bytes_fp32();
// tile: the member's (theta, phi) tile shape, 0: 8 x 32, 1: 16 x 16
int ens_fill_fp64(crn_grid* g, const void* U, void* R, int kchunk, int item0, double* nu, double* du, int tile,
                  void* dst);
int ens_fill_fp32(crn_grid* g, const void* U, void* R, int kchunk, int item0, double* nu, double* du, int tile,
                  void* dst);
// work items of a member for a tile shape and radial chunk
int ens_member_items(const crn_grid* g, int tile, int kchunk);
// the persistent launch over `nmem` member records of one tile shape
cudaError_t launch_ensemble_fp64(const void* dev, int nmem, int nitems, unsigned int* next, int limiter,
                                 int tile, int nctas, cudaStream_t st);
cudaError_t launch_ensemble_fp32(const void* dev, int nmem, int nitems, unsigned int* next, int limiter,
                                 int tile, int nctas, cudaStream_t st);
int ensemble_ctas_per_sm_fp64(int limiter, int tile);
int ensemble_ctas_per_sm_fp32(int limiter, int tile);
cudaError_t launch_ensemble_update(const void* dev, int nmem, int nitems, double cfl, bool fp32,
                                   cudaStream_t st);
size_t ens_update_bytes();
unsigned update_blocks(const crn_grid* g);
int update_blocks_per_sm(bool fp32);
void ens_update_fill(crn_grid* g, double* U64, int item0, int nitems, double* log_out, void* dst);
cudaError_t launch_efield_fp64(crn_grid* g, const double* U, double* E, bool volume, cudaStream_t st,
                                int* nl);
cudaError_t launch_efield_fp32(crn_grid* g, const float* U, double* E, bool volume, cudaStream_t st,
                                int* nl);

// shared-memory footprint of the tiled kernel for one precision
size_t tiled_smem_fp64();
size_t tiled_smem_fp32();
cudaError_t prepare_fp64();
cudaError_t prepare_fp32();

// record `msg` as the calling thread's last error (crn_last_error); returns code
int report_error(int code, const char* msg);

// resident CTAs per SM of the tiled kernel for this precision and limiter
// (after prepare_*), 0 on error
int tiled_ctas_per_sm_fp64(int limiter);
int tiled_ctas_per_sm_fp32(int limiter);
// the TMA-staged FP32 kernel: whether a shape tiles into its blocks, its
// block count, and its resident CTAs per SM
bool staged_shape_ok(int nt, int np);
int staged_tiles(int nt, int np);
int staged_ctas_per_sm_fp32(int limiter);

// Radial planes per CTA of the tiled kernel: the largest chunk count whose
// CTAs all fit in one wave of `slots` resident CTAs (fewer planes per CTA
// only add preamble work), at least 4 planes per CTA.
inline int choose_kchunk(int nr, long long ntiles, long long slots) {
  if (ntiles <= 0 || slots <= 0 || ntiles >= slots) return nr;
  long long nch = slots / ntiles;
  if (nch > nr) nch = nr;
  int kc = (int)((nr + nch - 1) / nch);
  return kc < 4 ? (nr < 4 ? nr : 4) : kc;
}

// Radial planes per CTA of the tiled kernel from a makespan model: the CTAs
// of each candidate chunk, in launch order (all tiles of chunk 0, then chunk
// 1, ...), are list-scheduled onto `slots` resident CTAs, each taking its
// planes plus `overhead` planes of preamble; the chunk with the shortest
// makespan wins (ties: the larger chunk).  Unlike one full wave, this lets
// the short last chunks run in the gaps the full ones leave (on 128 x 64 x 128:
// 14 planes, 288 full CTAs + 32 two-plane CTAs, beats 15 planes in one wave).
inline int choose_kchunk_balanced(int nr, long long ntiles, long long slots, int overhead = 3) {
  if (ntiles <= 0 || slots <= 0) return nr;
  const int kmin = nr < 4 ? nr : 4;
  int best = nr;
  long long best_t = -1;
  std::vector<long long> heap;
  for (int kc = nr; kc >= kmin; --kc) {
    const long long nch = (nr + kc - 1) / kc;
    const long long rem = nr - (nch - 1) * kc;
    const long long total = nch * ntiles;
    const long long S = slots < total ? slots : total;
    heap.assign((size_t)S, 0);  // slot free times (a min-heap)
    long long makespan = 0;
    for (long long y = 0; y < nch; ++y) {
      const long long dur = (y == nch - 1 ? rem : kc) + overhead;
      for (long long x = 0; x < ntiles; ++x) {
        std::pop_heap(heap.begin(), heap.end(), std::greater<long long>());
        const long long end = heap.back() + dur;
        heap.back() = end;
        std::push_heap(heap.begin(), heap.end(), std::greater<long long>());
        if (end > makespan) makespan = end;
      }
    }
    if (best_t < 0 || makespan < best_t) {
      best_t = makespan;
      best = kc;
    }
  }
  return best;
}

}  // namespace crn
