// ensemble.cu -- many independent shells (e.g. one per magnetogram) evaluated
// by one persistent launch of the tiled residual (residual_ensemble), and
// advanced by batched pseudo-time steps.
//
// Members are ordinary crn_grid objects of one precision and limiter and any
// sizes; the ensemble borrows them (they must outlive it) and keeps a device
// table of per-member records (geometry, physics, pointers, reduction
// scratch, work-item range, tile shape).  Work items are (member, tile,
// radial chunk); CTAs of the persistent grid take them from a counter, so the
// uneven sizes need no per-member launch and no host-side balancing.  Each
// member has a (theta, phi) tile shape (8 x 32 or 16 x 16) and a radial chunk
// (its own single-launch chunk by default); crn_ensemble_autotune picks both
// per size class from timed launches of that class's members.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "corona_internal.h"

struct crn_ensemble {
  std::vector<crn_grid*> g;
  int precision = 0, limiter = 0, device = 0;
  int kchunk = 0;          // last chunk set for all members (0: each member's own)
  std::vector<int> tile;   // per member: tile shape (0: 8 x 32, 1: 16 x 16)
  std::vector<int> kc;     // per member: radial chunk (0: the member's own)
  unsigned cfg_version = 1;  // bumped whenever tile or kc changes
  int nctas[crn::kEnsTileCount] = {};  // persistent grid per tile shape
  size_t msz = 0, usz = 0; // record sizes
  unsigned char* h_rec = nullptr;   // pinned residual records
  void* d_rec = nullptr;
  unsigned char* h_upd = nullptr;   // pinned update records
  void* d_upd = nullptr;
  unsigned int* next = nullptr;     // work-item counter per tile shape
  cudaEvent_t copied = nullptr;     // the last record upload has finished reading h_*
  int upd_items = 0;
  // the device table: member records grouped by tile shape
  int grp_off[crn::kEnsTileCount] = {}, grp_cnt[crn::kEnsTileCount] = {}, grp_items[crn::kEnsTileCount] = {};
  // what the device table holds now
  std::vector<const void*> kU;
  std::vector<void*> kR;
  double* kN = nullptr;
  double* kD = nullptr;
  unsigned kCfg = 0;          // cfg_version the table was built for
  const std::vector<int>* kSub = nullptr;  // member subset the table holds (nullptr: all)
  std::vector<double*> kU64;
  double* kLog = nullptr;
  bool upd_valid = false;
  int32_t last_launches = 0;
};

namespace {

int report(int code, const std::string& m) { return crn::report_error(code, m.c_str()); }

void free_ens(crn_ensemble* e) {
  if (!e) return;
  cudaFreeHost(e->h_rec);
  cudaFreeHost(e->h_upd);
  cudaFree(e->d_rec);
  cudaFree(e->d_upd);
  cudaFree(e->next);
  if (e->copied) cudaEventDestroy(e->copied);
  delete e;
}

int check_members_ready(const crn_ensemble* e) {
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != e->device) return report(CRN_E_ARG, "the current CUDA device is not the ensemble's device");
  for (size_t m = 0; m < e->g.size(); ++m)
    if (!e->g[m]->have_br)
      return report(CRN_E_STATE, "member " + std::to_string(m) + ": crn_set_inner_boundary has not been called");
  return CRN_OK;
}

int member_chunk(const crn_ensemble* e, int m) { return e->kc[m] > 0 ? e->kc[m] : e->g[m]->cfg.kchunk_tiled; }

// residual records for (U, R, norms, dtmin) with the members' tile shapes and
// radial chunks, for all members or only those in `sub` (U and R indexed by
// member); uploaded only if changed
int residual_records(crn_ensemble* e, const void* const* U, void* const* R, double* norms, double* dtmin,
                     cudaStream_t st, const std::vector<int>* sub = nullptr) {
  const int n = (int)e->g.size();
  bool same = sub == nullptr && e->kSub == nullptr && e->kCfg == e->cfg_version && e->kN == norms &&
              e->kD == dtmin && (int)e->kU.size() == n;
  for (int m = 0; same && m < n; ++m) same = e->kU[m] == U[m] && e->kR[m] == R[m];
  if (same) return CRN_OK;
  if (e->copied) cudaEventSynchronize(e->copied);  // h_rec may still be read by an earlier upload
  const int count = sub ? (int)sub->size() : n;
  int q = 0;  // records are grouped by tile shape, members in order within a group
  for (int t = 0; t < crn::kEnsTileCount; ++t) {
    e->grp_off[t] = q;
    int item0 = 0;
    for (int p = 0; p < count; ++p) {
      const int m = sub ? (*sub)[p] : p;
      if (e->tile[m] != t) continue;
      crn_grid* g = e->g[m];
      const int kc = member_chunk(e, m);
      if ((size_t)crn::ens_member_items(g, t, kc) > g->max_blocks)
        return report(CRN_E_ARG, "member " + std::to_string(m) + ": radial chunk " + std::to_string(kc) +
                                     " gives more work items than its reduction scratch holds");
      void* dst = e->h_rec + (size_t)q * e->msz;
      double* nu = norms ? norms + 9 * (size_t)m : nullptr;
      double* du = dtmin ? dtmin + m : nullptr;
      item0 += e->precision == CRN_FP64 ? crn::ens_fill_fp64(g, U[m], R[m], kc, item0, nu, du, t, dst)
                                        : crn::ens_fill_fp32(g, U[m], R[m], kc, item0, nu, du, t, dst);
      ++q;
    }
    e->grp_cnt[t] = q - e->grp_off[t];
    e->grp_items[t] = item0;
  }
  cudaError_t err = cudaMemcpyAsync(e->d_rec, e->h_rec, e->msz * count, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaEventRecord(e->copied, st);
  if (err != cudaSuccess) return report(CRN_E_CUDA, std::string("ensemble records: ") + cudaGetErrorString(err));
  e->kU.assign(U, U + n);
  e->kR.assign(R, R + n);
  e->kN = norms;
  e->kD = dtmin;
  e->kCfg = e->cfg_version;
  e->kSub = sub;
  if (sub) e->kU.clear();  // a subset table never matches a full call
  return CRN_OK;
}

int update_records(crn_ensemble* e, double* const* U64, double* log, cudaStream_t st) {
  const int n = (int)e->g.size();
  bool same = e->upd_valid && e->kLog == log && (int)e->kU64.size() == n;
  for (int m = 0; same && m < n; ++m) same = e->kU64[m] == U64[m];
  if (same) return CRN_OK;
  if (e->copied) cudaEventSynchronize(e->copied);
  int item0 = 0;
  for (int m = 0; m < n; ++m) {
    crn_grid* g = e->g[m];
    const int nb = (int)crn::update_blocks(g);
    crn::ens_update_fill(g, U64[m], item0, nb, log ? log + 9 * (size_t)m : nullptr, e->h_upd + (size_t)m * e->usz);
    item0 += nb;
  }
  cudaError_t err = cudaMemcpyAsync(e->d_upd, e->h_upd, e->usz * n, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaEventRecord(e->copied, st);
  if (err != cudaSuccess) return report(CRN_E_CUDA, std::string("ensemble records: ") + cudaGetErrorString(err));
  e->upd_items = item0;
  e->kU64.assign(U64, U64 + n);
  e->kLog = log;
  e->upd_valid = true;
  return CRN_OK;
}

// one persistent launch per tile shape in use; adds the launches to *count
cudaError_t launch(crn_ensemble* e, cudaStream_t st, int* count = nullptr) {
  for (int t = 0; t < crn::kEnsTileCount; ++t) {
    if (e->grp_cnt[t] == 0) continue;
    const void* rec = static_cast<const unsigned char*>(e->d_rec) + (size_t)e->grp_off[t] * e->msz;
    const cudaError_t err =
        e->precision == CRN_FP64
            ? crn::launch_ensemble_fp64(rec, e->grp_cnt[t], e->grp_items[t], e->next + t, e->limiter, t,
                                        e->nctas[t], st)
            : crn::launch_ensemble_fp32(rec, e->grp_cnt[t], e->grp_items[t], e->next + t, e->limiter, t,
                                        e->nctas[t], st);
    if (err != cudaSuccess) return err;
    if (count) ++*count;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

int crn_ensemble_create(crn_grid* const* grids, int32_t n, crn_ensemble** out) {
  if (!out) return report(CRN_E_ARG, "out is NULL");
  *out = nullptr;
  if (!grids || n < 1 || n > 4096) return report(CRN_E_ARG, "need 1 to 4096 member grids");
  for (int m = 0; m < n; ++m)
    if (!grids[m]) return report(CRN_E_ARG, "member " + std::to_string(m) + " is NULL");
  for (int m = 1; m < n; ++m) {
    if (grids[m]->d.precision != grids[0]->d.precision || grids[m]->d.limiter != grids[0]->d.limiter)
      return report(CRN_E_ARG, "members must share precision and limiter");
    if (grids[m]->device != grids[0]->device) return report(CRN_E_ARG, "members must share the device");
  }
  crn_ensemble* e = new crn_ensemble();
  e->g.assign(grids, grids + n);
  e->tile.assign(n, 0);
  e->kc.assign(n, 0);
  e->precision = grids[0]->d.precision;
  e->limiter = grids[0]->d.limiter;
  e->device = grids[0]->device;
  e->msz = e->precision == CRN_FP64 ? crn::ens_member_bytes_fp64() : crn::ens_member_bytes_fp32();
  e->usz = crn::ens_update_bytes();
  for (int t = 0; t < crn::kEnsTileCount; ++t) {
    const int per_sm = e->precision == CRN_FP64 ? crn::ensemble_ctas_per_sm_fp64(e->limiter, t)
                                                : crn::ensemble_ctas_per_sm_fp32(e->limiter, t);
    if (per_sm < 1) { free_ens(e); return report(CRN_E_CUDA, "ensemble kernel: no resident CTA fits"); }
    e->nctas[t] = per_sm * grids[0]->cfg.num_sms;
  }
  cudaError_t err = cudaMallocHost(&e->h_rec, e->msz * n);
  if (err == cudaSuccess) err = cudaMallocHost(&e->h_upd, e->usz * n);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_rec, e->msz * n);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_upd, e->usz * n);
  if (err == cudaSuccess) err = cudaMalloc(&e->next, crn::kEnsTileCount * sizeof(unsigned int));
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->copied, cudaEventDisableTiming);
  if (err != cudaSuccess) {
    free_ens(e);
    return report(CRN_E_CUDA, std::string("crn_ensemble_create: ") + cudaGetErrorString(err));
  }
  *out = e;
  return CRN_OK;
}

int crn_ensemble_destroy(crn_ensemble* e) {
  if (!e) return CRN_OK;
  cudaDeviceSynchronize();
  free_ens(e);
  return CRN_OK;
}

int crn_ensemble_set_kchunk(crn_ensemble* e, int32_t kchunk) {
  if (!e) return report(CRN_E_ARG, "ensemble is NULL");
  if (kchunk < 0 || kchunk > 4096) return report(CRN_E_ARG, "kchunk must be in [0, 4096]");
  e->kchunk = kchunk;
  e->kc.assign(e->g.size(), kchunk);
  ++e->cfg_version;
  return CRN_OK;
}

int crn_ensemble_set_member_config(crn_ensemble* e, int32_t m, int32_t tile, int32_t kchunk) {
  if (!e) return report(CRN_E_ARG, "ensemble is NULL");
  if (m < 0 || m >= (int)e->g.size()) return report(CRN_E_ARG, "member index out of range");
  if (tile < 0 || tile >= crn::kEnsTileCount) return report(CRN_E_ARG, "tile must be 0 (8 x 32) or 1 (16 x 16)");
  if (kchunk < 0 || kchunk > 4096) return report(CRN_E_ARG, "kchunk must be in [0, 4096]");
  e->tile[m] = tile;
  e->kc[m] = kchunk;
  ++e->cfg_version;
  return CRN_OK;
}

int crn_ensemble_member_config(const crn_ensemble* e, int32_t m, int32_t* tile, int32_t* kchunk) {
  if (!e) return report(CRN_E_ARG, "ensemble is NULL");
  if (m < 0 || m >= (int)e->g.size()) return report(CRN_E_ARG, "member index out of range");
  if (tile) *tile = e->tile[m];
  if (kchunk) *kchunk = member_chunk(e, m);
  return CRN_OK;
}

int32_t crn_ensemble_kchunk(const crn_ensemble* e) { return e ? e->kchunk : -1; }

int32_t crn_ensemble_launch_count(const crn_ensemble* e) { return e ? e->last_launches : 0; }

int crn_ensemble_residual(crn_ensemble* e, const void* const* U_dev, void* const* R_dev, double* norms9_dev,
                          double* dtmin_dev, void* stream) {
  if (!e) return report(CRN_E_ARG, "ensemble is NULL");
  if (!U_dev || !R_dev) return report(CRN_E_ARG, "U_dev and R_dev must not be NULL");
  int rc = check_members_ready(e);
  if (rc != CRN_OK) return rc;
  for (size_t m = 0; m < e->g.size(); ++m)
    if (!U_dev[m] || !R_dev[m] || U_dev[m] == R_dev[m])
      return report(CRN_E_ARG, "member " + std::to_string(m) + ": U and R must be distinct non-NULL buffers");
  cudaStream_t st = (cudaStream_t)stream;
  rc = residual_records(e, U_dev, R_dev, norms9_dev, dtmin_dev, st);
  if (rc != CRN_OK) return rc;
  int nl = 0;
  cudaError_t err = launch(e, st, &nl);
  e->last_launches = nl;
  if (err != cudaSuccess) return report(CRN_E_CUDA, std::string("crn_ensemble_residual: ") + cudaGetErrorString(err));
  return CRN_OK;
}

int crn_ensemble_pseudo_time_step(crn_ensemble* e, double* const* U64_dev, int32_t nsteps, double cfl,
                                  double* res_log10_dev, void* stream) {
  if (!e) return report(CRN_E_ARG, "ensemble is NULL");
  if (!U64_dev) return report(CRN_E_ARG, "U64_dev is NULL");
  if (nsteps < 0) return report(CRN_E_ARG, "nsteps must be >= 0");
  if (!(std::isfinite(cfl) && cfl > 0.0)) return report(CRN_E_ARG, "cfl must be > 0");
  int rc = check_members_ready(e);
  if (rc != CRN_OK) return rc;
  const int n = (int)e->g.size();
  for (int m = 0; m < n; ++m)
    if (!U64_dev[m]) return report(CRN_E_ARG, "member " + std::to_string(m) + ": U64 is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int launches = 0;
  std::vector<const void*> U(n);
  std::vector<void*> R(n);
  for (int m = 0; m < n; ++m) {
    crn_grid* g = e->g[m];
    U[m] = e->precision == CRN_FP64 ? (const void*)U64_dev[m] : (const void*)g->shadow;
    R[m] = g->rbuf;
  }
  rc = residual_records(e, U.data(), R.data(), nullptr, nullptr, st);
  if (rc == CRN_OK) rc = update_records(e, U64_dev, res_log10_dev, st);
  if (rc != CRN_OK) return rc;
  cudaError_t err = cudaSuccess;
  if (e->precision == CRN_FP32_BULK && nsteps > 0)
    for (int m = 0; m < n && err == cudaSuccess; ++m) {
      int nl = 0;
      err = crn::launch_shadow(e->g[m], U64_dev[m], st, &nl);
      launches += nl;
    }
  for (int s = 0; s < nsteps && err == cudaSuccess; ++s) {
    err = launch(e, st, &launches);
    if (err == cudaSuccess)
      err = crn::launch_ensemble_update(e->d_upd, n, e->upd_items, cfl, e->precision != CRN_FP64, st);
    ++launches;
  }
  e->last_launches = launches;
  if (err != cudaSuccess)
    return report(CRN_E_CUDA, std::string("crn_ensemble_pseudo_time_step: ") + cudaGetErrorString(err));
  return CRN_OK;
}

int crn_ensemble_autotune(crn_ensemble* e, const void* const* U_dev, void* const* R_dev, void* stream,
                          int32_t* kchunk_out) {
  if (!e) return report(CRN_E_ARG, "ensemble is NULL");
  if (!U_dev || !R_dev) return report(CRN_E_ARG, "U_dev and R_dev must not be NULL");
  int rc = check_members_ready(e);
  if (rc != CRN_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)e->g.size();
  // size classes: members with the same (n_theta, n_phi), in order of first appearance
  std::vector<std::vector<int>> classes;
  std::vector<std::pair<int, int>> keys;
  for (int m = 0; m < n; ++m) {
    const std::pair<int, int> key(e->g[m]->shape.nt, e->g[m]->shape.np);
    size_t c = 0;
    while (c < keys.size() && keys[c] != key) ++c;
    if (c == keys.size()) {
      keys.push_back(key);
      classes.emplace_back();
    }
    classes[c].push_back(m);
  }
  static const int cand[] = {0, 4, 6, 8, 12, 16, 24, 32, 48};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int launches = 0, big_class = 0;
  int64_t big_cells = -1;
  std::vector<int> best_k(classes.size(), 0);
  for (size_t c = 0; c < classes.size(); ++c) {
    const std::vector<int>& mem = classes[c];
    int nr_max = 0;
    int64_t cells = 0;
    for (int m : mem) {
      nr_max = std::max(nr_max, e->g[m]->shape.nr);
      cells += e->g[m]->shape.ncell;
    }
    if (cells > big_cells) { big_cells = cells; big_class = (int)c; }
    float best_ms = INFINITY;
    int best_tile = 0, bestk = 0;
    for (int tile = 0; tile < crn::kEnsTileCount; ++tile)
      for (int k : cand) {
        if (k > 0 && k > nr_max) continue;
        for (int m : mem) { e->tile[m] = tile; e->kc[m] = k; }
        ++e->cfg_version;
        rc = residual_records(e, U_dev, R_dev, nullptr, nullptr, st, &mem);
        if (rc != CRN_OK) continue;  // this chunk overflows a member's scratch
        int nl = 0;
        cudaError_t err = launch(e, st, &nl);  // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(a, st);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch(e, st, &nl);
        if (err == cudaSuccess) err = cudaEventRecord(b, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
        if (err != cudaSuccess) {
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return report(CRN_E_CUDA, std::string("crn_ensemble_autotune: ") + cudaGetErrorString(err));
        }
        launches += nl;
        if (ms < best_ms) { best_ms = ms; best_tile = tile; bestk = k; }
      }
    if (!(best_ms < INFINITY)) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return report(CRN_E_ARG, "no radial chunk fits the reduction scratch of every member of a size class");
    }
    for (int m : mem) { e->tile[m] = best_tile; e->kc[m] = bestk; }
    best_k[c] = bestk;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ++e->cfg_version;
  e->kSub = nullptr;
  e->kU.clear();  // the next call rebuilds the full table
  e->kchunk = best_k[big_class];
  if (kchunk_out) *kchunk_out = e->kchunk;
  e->last_launches = launches;
  return CRN_OK;
}

}  // extern "C"
