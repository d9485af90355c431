// corona_api.cu -- the C ABI of libcorona (declared in include/corona.h):
// grid set-up (validation, exact shell geometry, device buffers), argument
// checks, kernel launches and error reporting.
//
// Geometry (arXiv 2209.04481 uses an unstructured prism mesh, Sect. 2.1; this
// library uses a structured (r, theta, phi) shell over the same domain): the
// face-area vectors are the exact integrals of the unit normal over each face,
//   r face      S = r^2 (X 2 sin(dphi/2) cos phi_c, X 2 sin(dphi/2) sin phi_c, Z dphi),
//               X = (dtheta - cos(t1 + t2) sin dtheta) / 2, Z = sin(t1 + t2) sin(dtheta) / 2,
//   theta face  S = (r2^2 - r1^2)/2 sin t (cos t 2 sin(dphi/2) cos phi_c,
//                                          cos t 2 sin(dphi/2) sin phi_c, -sin t dphi),
//   phi face    S = (r2^2 - r1^2)/2 dtheta (-sin phi, cos phi, 0),
// and the volumes V = (r2^3 - r1^3)/3 (cos t1 - cos t2) dphi, so that every
// cell closes (sum of outward S = 0) and a uniform state is preserved.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "corona_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(CRN_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

const double kPi = 3.14159265358979323846;

bool finite(double x) { return std::isfinite(x); }

int validate(const crn_grid_desc* d) {
  if (!d) return fail(CRN_E_ARG, "crn_grid_desc is NULL");
  if (d->n_r < 2) return fail(CRN_E_ARG, "n_r must be >= 2");
  if (d->n_theta < 2) return fail(CRN_E_ARG, "n_theta must be >= 2");
  if (d->n_phi < 8 || d->n_phi % 8 != 0) return fail(CRN_E_ARG, "n_phi must be a positive multiple of 8");
  const double ncell = (double)d->n_r * d->n_theta * d->n_phi;
  if (ncell > 2.0e9) return fail(CRN_E_ARG, "grid has more than 2e9 cells");
  if (d->precision != CRN_FP64 && d->precision != CRN_FP32_BULK)
    return fail(CRN_E_ARG, "precision must be CRN_FP64 or CRN_FP32_BULK");
  if (d->limiter < CRN_LIM_NONE || d->limiter > CRN_LIM_VANALBADA)
    return fail(CRN_E_ARG, "unknown limiter");
  if (d->kernel != CRN_KERNEL_TILED && d->kernel != CRN_KERNEL_CELLWISE && d->kernel != CRN_KERNEL_TILED_REGS &&
      d->kernel != CRN_KERNEL_STAGED)
    return fail(CRN_E_ARG, "unknown kernel variant");
  if (!(finite(d->r_in) && finite(d->r_out) && d->r_in > 0.0 && d->r_out > d->r_in))
    return fail(CRN_E_ARG, "need 0 < r_in < r_out");
  if (!(finite(d->gamma) && d->gamma > 1.0)) return fail(CRN_E_ARG, "gamma must be > 1");
  if (!(finite(d->c_h) && d->c_h >= 0.0)) return fail(CRN_E_ARG, "c_h must be >= 0");
  if (!finite(d->g0)) return fail(CRN_E_ARG, "g0 must be finite");
  if (!(finite(d->lim_eps) && d->lim_eps >= 0.0)) return fail(CRN_E_ARG, "lim_eps must be >= 0");
  // the smooth van Albada form is 0/0 where both one-sided slopes vanish
  if (d->limiter == CRN_LIM_VANALBADA && !(d->lim_eps > 0.0))
    return fail(CRN_E_ARG, "lim_eps must be > 0 with the van Albada limiter");
  if (!finite(d->outer_rho_exp) || !finite(d->outer_br_exp))
    return fail(CRN_E_ARG, "outer exponents must be finite");
  if (!(finite(d->rho_b) && d->rho_b > 0.0 && finite(d->p_b) && d->p_b > 0.0))
    return fail(CRN_E_ARG, "rho_b and p_b must be > 0");
  if (d->inner_bc < CRN_INNER_LOW_E || d->inner_bc > CRN_INNER_LOW_E_WP)
    return fail(CRN_E_ARG, "unknown inner_bc");
  if ((d->outer_vr_mass != 0 && d->outer_vr_mass != 1) ||
      (d->outer_psi_extrap != 0 && d->outer_psi_extrap != 1) || d->reserved_ != 0)
    return fail(CRN_E_ARG, "outer_vr_mass / outer_psi_extrap must be 0 or 1, reserved_ 0");
  if (!finite(d->vr_star) || !finite(d->outer_bphi_exp) || !finite(d->outer_vphi_exp))
    return fail(CRN_E_ARG, "vr_star and the outer exponents must be finite");
  if (d->r_last != 0.0 && !(finite(d->r_last) && d->r_last > d->r_in && d->r_last < d->r_out))
    return fail(CRN_E_ARG, "r_last must be 0 or in (r_in, r_out)");
  if (!(finite(d->psi_damp) && d->psi_damp >= 0.0)) return fail(CRN_E_ARG, "psi_damp must be >= 0");
  return CRN_OK;
}

// Host geometry in FP64 (layout documented on crn::Geo).
struct HostGeo {
  std::vector<double> ra, rb, rv, inv_dm, inv_dp, hm, hp, grav, ar, at, av, nr, nth, nph, rhat;
  double dtheta = 0, fa = 1, fb = 1, fbp = 1, fvr = 1, fvp = 1;
};

HostGeo build_geometry(const crn_grid_desc& d) {
  HostGeo h;
  const int nr = d.n_r, nt = d.n_theta, np = d.n_phi;
  std::vector<double> rf(nr + 1), rc(nr);
  // geometric faces over M cells up to r_top; a set r_last keeps one thin
  // outermost cell [r_last, r_out] (the mesh of Sect. 4.3)
  const bool thin = d.r_last != 0.0;
  const int M = thin ? nr - 1 : nr;
  const double r_top = thin ? d.r_last : d.r_out;
  for (int k = 0; k <= M; ++k) rf[k] = d.r_in * std::pow(r_top / d.r_in, (double)k / M);
  rf[0] = d.r_in;
  rf[M] = r_top;
  rf[nr] = d.r_out;
  for (int k = 0; k < nr; ++k) rc[k] = 0.5 * (rf[k] + rf[k + 1]);
  const double rc_in = 2.0 * d.r_in - rc[0];            // mirrored ghost centres
  const double rc_out = 2.0 * d.r_out - rc[nr - 1];
  h.ra.resize(nr + 1);
  for (int k = 0; k <= nr; ++k) h.ra[k] = rf[k] * rf[k];
  h.rb.resize(nr); h.rv.resize(nr); h.inv_dm.resize(nr); h.inv_dp.resize(nr);
  h.hm.resize(nr); h.hp.resize(nr); h.grav.resize(nr);
  for (int k = 0; k < nr; ++k) {
    const double r1 = rf[k], r2 = rf[k + 1];
    h.rb[k] = 0.5 * (r2 - r1) * (r2 + r1);
    h.rv[k] = (r2 - r1) * (r2 * r2 + r2 * r1 + r1 * r1) / 3.0;
    const double cm = k == 0 ? rc_in : rc[k - 1];
    const double cp = k == nr - 1 ? rc_out : rc[k + 1];
    h.inv_dm[k] = 1.0 / (rc[k] - cm);
    h.inv_dp[k] = 1.0 / (cp - rc[k]);
    h.hm[k] = rc[k] - r1;
    h.hp[k] = r2 - rc[k];
    h.grav[k] = d.g0 / (rc[k] * rc[k]);
  }
  const double dth = kPi / nt, dph = 2.0 * kPi / np;
  const double s2 = 2.0 * std::sin(0.5 * dph);
  h.dtheta = dth;
  h.ar.resize(nt); h.av.resize(nt); h.at.assign(nt + 1, 0.0);
  h.nr.assign((size_t)3 * nt * np, 0.0);
  h.rhat.assign((size_t)3 * nt * np, 0.0);
  h.nth.assign((size_t)3 * (nt + 1) * np, 0.0);
  h.nph.assign((size_t)2 * np, 0.0);
  const size_t cs = (size_t)nt * np, ts = (size_t)(nt + 1) * np;
  for (int j = 0; j < nt; ++j) {
    const double t1 = j * dth, t2 = (j + 1) * dth, tc = (j + 0.5) * dth;
    const double X = 0.5 * (dth - std::cos(t1 + t2) * std::sin(dth));
    const double Z = 0.5 * std::sin(t1 + t2) * std::sin(dth);
    h.ar[j] = std::sqrt(X * X * s2 * s2 + Z * Z * dph * dph);
    h.av[j] = 2.0 * std::sin(tc) * std::sin(0.5 * dth) * dph;
    for (int i = 0; i < np; ++i) {
      const double pc = (i + 0.5) * dph;
      const size_t c = (size_t)j * np + i;
      h.nr[c] = X * s2 * std::cos(pc) / h.ar[j];
      h.nr[cs + c] = X * s2 * std::sin(pc) / h.ar[j];
      h.nr[2 * cs + c] = Z * dph / h.ar[j];
      h.rhat[c] = std::sin(tc) * std::cos(pc);
      h.rhat[cs + c] = std::sin(tc) * std::sin(pc);
      h.rhat[2 * cs + c] = std::cos(tc);
    }
  }
  for (int jf = 1; jf < nt; ++jf) {  // pole faces (jf = 0, nt) keep zero area
    const double t = jf * dth, st = std::sin(t), ct = std::cos(t);
    h.at[jf] = st * std::sqrt(ct * ct * s2 * s2 + st * st * dph * dph);
    for (int i = 0; i < np; ++i) {
      const double pc = (i + 0.5) * dph;
      const size_t c = (size_t)jf * np + i;
      h.nth[c] = st * ct * s2 * std::cos(pc) / h.at[jf];
      h.nth[ts + c] = st * ct * s2 * std::sin(pc) / h.at[jf];
      h.nth[2 * ts + c] = -st * st * dph / h.at[jf];
    }
  }
  for (int i = 0; i < np; ++i) {
    const double p = i * dph;
    h.nph[i] = -std::sin(p);
    h.nph[np + i] = std::cos(p);
  }
  const double rI = rc[nr - 1], rG = 2.0 * d.r_out - rI;
  h.fa = std::pow(rI / rG, d.outer_rho_exp);
  h.fb = std::pow(rI / rG, d.outer_br_exp);
  h.fbp = std::pow(rI / rG, d.outer_bphi_exp);
  h.fvr = d.outer_vr_mass ? std::pow(rI / rG, 2.0 - d.outer_rho_exp) : 1.0;  // V_r r^2 rho = const
  h.fvp = std::pow(rI / rG, d.outer_vphi_exp);
  return h;
}

// upload the geometry as one allocation of T and carve it into arrays
template <class T>
int upload_geometry(const HostGeo& h, crn::GeoBuf<T>& out) {
  const std::vector<double>* parts[] = {&h.ra, &h.rb, &h.rv, &h.inv_dm, &h.inv_dp, &h.hm, &h.hp,
                                        &h.grav, &h.ar, &h.at, &h.av, &h.nr, &h.nth, &h.nph,
                                        &h.rhat};
  const int nparts = sizeof(parts) / sizeof(parts[0]);
  size_t total = 0;
  std::vector<size_t> off(nparts);
  for (int q = 0; q < nparts; ++q) {
    off[q] = total;
    total += (parts[q]->size() + 31) & ~size_t(31);  // 256-byte aligned sub-arrays
  }
  std::vector<T> host(total, (T)0);
  for (int q = 0; q < nparts; ++q)
    for (size_t e = 0; e < parts[q]->size(); ++e) host[off[q] + e] = (T)(*parts[q])[e];
  T* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, total * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(geometry)");
  e = cudaMemcpy(dev, host.data(), total * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(dev); return cuda_fail(e, "cudaMemcpy(geometry)"); }
  out.base = dev;
  crn::Geo<T>& g = out.geo;
  const T* p[15];
  for (int q = 0; q < nparts; ++q) p[q] = dev + off[q];
  g.ra = p[0]; g.rb = p[1]; g.rv = p[2]; g.inv_dm = p[3]; g.inv_dp = p[4]; g.hm = p[5];
  g.hp = p[6]; g.grav = p[7]; g.ar = p[8]; g.at = p[9]; g.av = p[10]; g.nr = p[11];
  g.nth = p[12]; g.nph = p[13]; g.rhat = p[14];
  g.dtheta = (T)h.dtheta;
  return CRN_OK;
}

template <class T>
crn::Phys<T> make_phys(const crn_grid_desc& d, const HostGeo& h) {
  const double fa = h.fa, fb = h.fb;
  crn::Phys<T> ph;
  ph.gamma = (T)d.gamma;
  ph.gm1 = (T)(d.gamma - 1.0);
  ph.igm1 = (T)(1.0 / (d.gamma - 1.0));
  ph.ch = (T)d.c_h;
  ph.ch2 = (T)(d.c_h * d.c_h);
  ph.eps = (T)d.lim_eps;
  ph.rho_b = (T)d.rho_b;
  ph.p_b = (T)d.p_b;
  ph.fa = (T)fa;
  ph.fb = (T)fb;
  ph.fbp = (T)h.fbp;
  ph.fvr = (T)h.fvr;
  ph.fvp = (T)h.fvp;
  ph.psi_out = d.outer_psi_extrap ? (T)1 : (T)-1;
  ph.psi_damp = (T)d.psi_damp;
  ph.inner_bc = d.inner_bc;
  ph.vr_star = d.vr_star;
  return ph;
}

void free_grid(crn_grid* g) {
  if (!g) return;
  cudaFree(g->g64.base);
  cudaFree(g->g32.base);
  cudaFree(g->br);
  cudaFree(g->partials);
  cudaFree(g->counter);
  cudaFree(g->stats);
  cudaFree(g->err_flags);
  cudaFree(g->err_cell);
  cudaFree(g->rbuf);
  cudaFree(g->shadow);
  cudaFree(g->vjp_buf);
  crn::nk_free(g->nk);
  crn::host_pipe_free(g->pipe);
  delete g;
}

size_t elem_size(const crn_grid* g) { return g->d.precision == CRN_FP64 ? 8 : 4; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_ready(const crn_grid* g) {
  if (!g) return fail(CRN_E_ARG, "grid is NULL");
  if (!g->have_br) return fail(CRN_E_STATE, "crn_set_inner_boundary has not been called");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return fail(CRN_E_ARG, "the current CUDA device is not the grid's device");
  return CRN_OK;
}

// as check_ready, for calls that do not read the inner boundary values
int check_ready_u(const crn_grid* g) {
  if (!g) return fail(CRN_E_ARG, "grid is NULL");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return fail(CRN_E_ARG, "the current CUDA device is not the grid's device");
  return CRN_OK;
}

int efield(crn_grid* g, const void* U, double* E, bool volume, void* stream) {
  int nl = 0;
  cudaError_t e = g->d.precision == CRN_FP64
                      ? crn::launch_efield_fp64(g, (const double*)U, E, volume, (cudaStream_t)stream, &nl)
                      : crn::launch_efield_fp32(g, (const float*)U, E, volume, (cudaStream_t)stream, &nl);
  g->last_launches = nl;
  if (e != cudaSuccess) return cuda_fail(e, volume ? "crn_efield launch" : "crn_boundary_efield launch");
  return CRN_OK;
}

}  // namespace

namespace crn {
int report_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }
}  // namespace crn

extern "C" {

int crn_grid_desc_default(crn_grid_desc* d, int32_t n_r, int32_t n_theta, int32_t n_phi) {
  if (!d) return fail(CRN_E_ARG, "crn_grid_desc is NULL");
  std::memset(d, 0, sizeof(*d));
  d->n_r = n_r;
  d->n_theta = n_theta;
  d->n_phi = n_phi;
  d->precision = CRN_FP32_BULK;
  d->limiter = CRN_LIM_VANALBADA;
  d->kernel = CRN_KERNEL_TILED;
  d->r_in = 1.0;
  d->r_out = 21.5;
  d->gamma = 1.05;
  d->c_h = 1.0;
  // G M_sun / (R_sun V_ref^2), V_ref = B_ref / sqrt(mu0 rho_ref) (Sect. 2.1 values)
  const double vref = 2.2e-4 / std::sqrt(4e-7 * kPi * 1.67e-13);
  d->g0 = 1.3271244e20 / (6.957e8 * vref * vref);
  d->lim_eps = 1e-12;
  d->outer_rho_exp = 2.0;
  d->outer_br_exp = 2.0;
  d->rho_b = 1.0;
  d->p_b = d->g0 / 10.0;  // isothermal wind with its sonic point at 5 R_sun
  d->inner_bc = CRN_INNER_LOW_E;
  d->vr_star = 1935.07 / vref;  // Wind-Predict's inner outflow (Sect. 3.2), large-E only
  return CRN_OK;
}

int32_t crn_tiled_radial_chunk(int32_t n_r, int64_t ntiles, int64_t slots, int32_t overhead) {
  if (n_r < 1 || ntiles < 1 || slots < 1 || overhead < 0) return -1;
  return crn::choose_kchunk_balanced(n_r, ntiles, slots, overhead);
}

int crn_grid_create(const crn_grid_desc* d, crn_grid** out) {
  if (!out) return fail(CRN_E_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(d);
  if (rc != CRN_OK) return rc;
  crn_grid* g = new crn_grid();
  g->d = *d;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaGetDevice"); }
  g->shape.nr = d->n_r;
  g->shape.nt = d->n_theta;
  g->shape.np = d->n_phi;
  g->shape.ncell = (int64_t)d->n_r * d->n_theta * d->n_phi;
  const HostGeo h = build_geometry(*d);
  g->ph64 = make_phys<double>(*d, h);
  g->ph32 = make_phys<float>(*d, h);
  // opt the kernels in to their shared memory, then size the tiled launch:
  // radial chunk from the makespan model over the resident CTA slots
  e = d->precision == CRN_FP64 ? crn::prepare_fp64() : crn::prepare_fp32();
  if (e != cudaSuccess) { delete g; return cuda_fail(e, "kernel attributes"); }
  {
    const int tt = 8, tp = 32;
    const int64_t ntiles = (int64_t)((d->n_theta + tt - 1) / tt) * ((d->n_phi + tp - 1) / tp);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device);
    const int per_sm = d->precision == CRN_FP64 ? crn::tiled_ctas_per_sm_fp64(d->limiter)
                                                 : crn::tiled_ctas_per_sm_fp32(d->limiter);
    int kc = crn::choose_kchunk_balanced(d->n_r, ntiles, (long long)std::max(nsm, 1) * std::max(per_sm, 1));
    if (const char* env = std::getenv("CRN_KCHUNK")) {  // tuning override
      const int v = std::atoi(env);
      if (v >= 1) kc = v;
    }
    g->cfg.kchunk_tiled = kc;
    g->cfg.num_sms = std::max(nsm, 1);
    g->cfg.update_per_sm = crn::update_blocks_per_sm(d->precision != CRN_FP64);
    int64_t tiled_blocks = ntiles * ((d->n_r + kc - 1) / kc);
    // the TMA-staged FP32 kernel, on request: whole 8 x 32 blocks only
    if (d->precision == CRN_FP32_BULK && d->kernel == CRN_KERNEL_STAGED &&
        crn::staged_shape_ok(d->n_theta, d->n_phi)) {
      const int sper = crn::staged_ctas_per_sm_fp32(d->limiter);
      if (sper > 0) {
        const int64_t st = crn::staged_tiles(d->n_theta, d->n_phi);
        int kcs = crn::choose_kchunk_balanced(d->n_r, st, (long long)std::max(nsm, 1) * sper);
        if (const char* env = std::getenv("CRN_KCHUNK")) {
          const int v = std::atoi(env);
          if (v >= 1) kcs = v;
        }
        g->cfg.staged = true;
        g->cfg.kchunk_staged = kcs;
        tiled_blocks = std::max<int64_t>(tiled_blocks, st * ((d->n_r + kcs - 1) / kcs));
      }
    }
    const int64_t cell_blocks = (g->shape.ncell + 255) / 256;
    g->max_blocks = (size_t)std::max<int64_t>(std::max<int64_t>(tiled_blocks, cell_blocks), 4 * 152 * 8);
  }
  rc = upload_geometry(h, g->g64);
  if (rc == CRN_OK) rc = upload_geometry(h, g->g32);
  if (rc != CRN_OK) { free_grid(g); return rc; }
  const size_t nt_np = (size_t)d->n_theta * d->n_phi * (d->inner_bc == CRN_INNER_LARGE_E ? 2 : 1);
  const size_t n9 = (size_t)9 * g->shape.ncell;
  struct { void** p; size_t bytes; const char* what; } allocs[] = {
      {(void**)&g->br, nt_np * sizeof(double), "B_r"},
      {(void**)&g->partials, g->max_blocks * crn::RED_STRIDE * sizeof(double), "partials"},
      {(void**)&g->counter, sizeof(unsigned int), "counter"},
      {(void**)&g->stats, 32 * sizeof(double), "stats"},
      {(void**)&g->err_flags, sizeof(unsigned int), "error flags"},
      {(void**)&g->err_cell, sizeof(unsigned long long), "error cell"},
      {(void**)&g->rbuf, n9 * elem_size(g), "residual scratch"},
  };
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) { free_grid(g); return cuda_fail(e, a.what); }
  }
  if (d->precision == CRN_FP32_BULK) {
    e = cudaMalloc(&g->shadow, n9 * sizeof(float));
    if (e != cudaSuccess) { free_grid(g); return cuda_fail(e, "FP32 shadow"); }
  }
  cudaMemset(g->counter, 0, sizeof(unsigned int));
  cudaMemset(g->stats, 0, 32 * sizeof(double));
  cudaMemset(g->err_flags, 0, sizeof(unsigned int));
  cudaMemset(g->err_cell, 0xff, sizeof(unsigned long long));
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { free_grid(g); return cuda_fail(e, "grid set-up"); }
  *out = g;
  return CRN_OK;
}

int crn_grid_destroy(crn_grid* g) {
  if (!g) return CRN_OK;
  cudaDeviceSynchronize();
  free_grid(g);
  return CRN_OK;
}

int crn_set_inner_boundary(crn_grid* g, const double* Br_dev, void* stream) {
  if (!g) return fail(CRN_E_ARG, "grid is NULL");
  if (!Br_dev || !is_device_ptr(Br_dev)) return fail(CRN_E_ARG, "Br_dev must be a device pointer");
  const size_t bytes = (size_t)g->d.n_theta * g->d.n_phi * sizeof(double) *
                       (g->d.inner_bc == CRN_INNER_LARGE_E ? 2 : 1);
  cudaError_t e = cudaMemcpyAsync(g->br, Br_dev, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "crn_set_inner_boundary");
  g->have_br = true;
  return CRN_OK;
}

int crn_residual(crn_grid* g, const void* U_dev, void* R_dev, double* norms9_dev, double* dtmin_dev,
                 void* stream) {
  int rc = check_ready(g);
  if (rc != CRN_OK) return rc;
  if (!U_dev || !R_dev) return fail(CRN_E_ARG, "U_dev and R_dev must not be NULL");
  const size_t bytes = (size_t)9 * g->shape.ncell * elem_size(g);
  const char* a = (const char*)U_dev;
  const char* b = (const char*)R_dev;
  if (a < b + bytes && b < a + bytes) return fail(CRN_E_ARG, "U_dev and R_dev overlap");
  if (!is_device_ptr(U_dev) || !is_device_ptr(R_dev))
    return fail(CRN_E_ARG, "U_dev and R_dev must be device pointers");
  if ((norms9_dev && !is_device_ptr(norms9_dev)) || (dtmin_dev && !is_device_ptr(dtmin_dev)))
    return fail(CRN_E_ARG, "norms9_dev / dtmin_dev must be device pointers");
  int nl = 0;
  cudaError_t e;
  if (g->d.precision == CRN_FP64)
    e = crn::launch_residual_fp64(g, (const double*)U_dev, (double*)R_dev, norms9_dev, dtmin_dev,
                                  (cudaStream_t)stream, &nl);
  else
    e = crn::launch_residual_fp32(g, (const float*)U_dev, (float*)R_dev, norms9_dev, dtmin_dev,
                                  (cudaStream_t)stream, &nl);
  g->last_launches = nl;
  if (e != cudaSuccess) return cuda_fail(e, "crn_residual launch");
  return CRN_OK;
}

int crn_residual_vjp(crn_grid* g, const void* U_dev, const void* Rbar_dev, void* Ubar_dev,
                     double* Brbar_dev, void* stream) {
  int rc = check_ready(g);
  if (rc != CRN_OK) return rc;
  if (!U_dev || !Rbar_dev || !Ubar_dev) return fail(CRN_E_ARG, "U_dev, Rbar_dev and Ubar_dev must not be NULL");
  const size_t bytes = (size_t)9 * g->shape.ncell * elem_size(g);
  const char* u = (const char*)U_dev;
  const char* rb = (const char*)Rbar_dev;
  const char* ub = (const char*)Ubar_dev;
  if ((ub < u + bytes && u < ub + bytes) || (ub < rb + bytes && rb < ub + bytes))
    return fail(CRN_E_ARG, "Ubar_dev overlaps U_dev or Rbar_dev");
  if (!is_device_ptr(U_dev) || !is_device_ptr(Rbar_dev) || !is_device_ptr(Ubar_dev) ||
      (Brbar_dev && !is_device_ptr(Brbar_dev)))
    return fail(CRN_E_ARG, "VJP arguments must be device pointers");
  if (!g->vjp_buf && crn::vjp_scratch_bytes(g) > 0) {  // first VJP call: face-contribution scratch
    cudaError_t e = cudaMalloc(&g->vjp_buf, crn::vjp_scratch_bytes(g));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(VJP scratch)");
  }
  int nl = 0;
  cudaError_t e;
  if (g->d.precision == CRN_FP64)
    e = crn::launch_vjp_fp64(g, (const double*)U_dev, (const double*)Rbar_dev, (double*)Ubar_dev,
                             Brbar_dev, (cudaStream_t)stream, &nl);
  else
    e = crn::launch_vjp_fp32(g, (const float*)U_dev, (const float*)Rbar_dev, (float*)Ubar_dev,
                             Brbar_dev, (cudaStream_t)stream, &nl);
  g->last_launches = nl;
  if (e != cudaSuccess) return cuda_fail(e, "crn_residual_vjp launch");
  return CRN_OK;
}

int crn_pseudo_time_step(crn_grid* g, double* U64_dev, int32_t nsteps, double cfl,
                         double* res_log10_dev, void* stream) {
  int rc = check_ready(g);
  if (rc != CRN_OK) return rc;
  if (!U64_dev || !is_device_ptr(U64_dev)) return fail(CRN_E_ARG, "U64_dev must be a device pointer");
  if (nsteps < 0) return fail(CRN_E_ARG, "nsteps must be >= 0");
  if (!(std::isfinite(cfl) && cfl > 0.0)) return fail(CRN_E_ARG, "cfl must be > 0");
  if (res_log10_dev && !is_device_ptr(res_log10_dev))
    return fail(CRN_E_ARG, "res_log10_dev must be a device pointer");
  cudaStream_t st = (cudaStream_t)stream;
  int total = 0, nl = 0;
  cudaError_t e = cudaSuccess;
  if (g->d.precision == CRN_FP32_BULK && nsteps > 0) {
    e = crn::launch_shadow(g, U64_dev, st, &nl);
    total += nl;
  }
  for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
    if (g->d.precision == CRN_FP64)
      e = crn::launch_residual_fp64(g, U64_dev, (double*)g->rbuf, nullptr, nullptr, st, &nl);
    else
      e = crn::launch_residual_fp32(g, g->shadow, (float*)g->rbuf, nullptr, nullptr, st, &nl);
    total += nl;
    if (e != cudaSuccess) break;
    e = crn::launch_update(g, U64_dev, cfl, res_log10_dev ? res_log10_dev + 9 * (size_t)s : nullptr,
                           st, &nl);
    total += nl;
  }
  g->last_launches = total;
  if (e != cudaSuccess) return cuda_fail(e, "crn_pseudo_time_step launch");
  return CRN_OK;
}

int crn_boundary_efield(crn_grid* g, const void* U_dev, double* E_dev, void* stream) {
  int rc = check_ready(g);
  if (rc != CRN_OK) return rc;
  if (!U_dev || !E_dev || !is_device_ptr(U_dev) || !is_device_ptr(E_dev))
    return fail(CRN_E_ARG, "U_dev and E_dev must be device pointers");
  return efield(g, U_dev, E_dev, false, stream);
}

int crn_efield(crn_grid* g, const void* U_dev, double* E_dev, void* stream) {
  int rc = check_ready_u(g);
  if (rc != CRN_OK) return rc;
  if (!U_dev || !E_dev || !is_device_ptr(U_dev) || !is_device_ptr(E_dev))
    return fail(CRN_E_ARG, "U_dev and E_dev must be device pointers");
  return efield(g, U_dev, E_dev, true, stream);
}

int crn_sync_status(crn_grid* g, void* stream) {
  if (!g) return fail(CRN_E_ARG, "grid is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned int flags = 0;
  unsigned long long cell = ~0ull;
  e = cudaMemcpy(&flags, g->err_flags, sizeof(flags), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&cell, g->err_cell, sizeof(cell), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->err_flags, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(g->err_cell, 0xff, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "crn_sync_status");
  g->last_bad_cell = (flags & 1u) ? (int64_t)cell : -1;
  if (flags & 2u) return fail(CRN_E_TIMEOUT, "a kernel's bounded wait for an asynchronous copy gave up");
  if (flags) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "non-physical or non-finite state at cell %lld",
                  (long long)g->last_bad_cell);
    return fail(CRN_E_NONPHYSICAL, buf);
  }
  g_last_error.clear();
  return CRN_OK;
}

int64_t crn_last_bad_cell(const crn_grid* g) { return g ? g->last_bad_cell : -1; }

const char* crn_last_error(void) { return g_last_error.c_str(); }

int32_t crn_last_launch_count(const crn_grid* g) { return g ? g->last_launches : 0; }

int32_t crn_last_kernel(const crn_grid* g) { return g ? g->last_kernel : -1; }

}  // extern "C"
