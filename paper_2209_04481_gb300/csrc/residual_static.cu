// residual_static.cu -- crn_residual_static: one residual evaluation that
// allocates nothing.
//
// Some callers cannot allocate device memory: code running inside a memory
// budget fixed by a host framework, plugins whose host forbids cudaMalloc
// during a solve, or callers that must not trigger an allocator's implicit
// device synchronisation.  For them this entry point evaluates the same
// residual as crn_residual (the same tiled kernel) without a crn_grid: the
// exact shell geometry, the reduction partials, the CTA arrival counter and
// the error word live in one file-scope device array of fixed size, which
// every GPU that loads the library holds until the process exits.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress and opts the kernels in to
// their shared memory; make that first call before any stream capture.  When
// the descriptor differs from the one the geometry was last built for, the
// geometry is rebuilt on the device, on the caller's stream, before the
// residual kernel.  A call recorded in a CUDA graph records the geometry build
// with it; after that, every call on the device rebuilds the geometry, since a
// replay may have overwritten it.  All calls share the array and it keeps the last call's
// contents: calls whose kernels overlap on the GPU (two streams, two host
// threads) race on it and must be serialised by the caller.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "corona_internal.h"
#include "residual.cuh"

namespace {

// limits of the shared array
constexpr int kMaxNr = 1024;
constexpr int kMaxNt = 1024;
constexpr int kMaxNp = 2048;
constexpr int kMaxCols = 32768;   // n_theta * n_phi
constexpr int kMaxBlocks = 8192;  // CTAs of one launch (reduction partials)
constexpr int kMaxDevices = 64;

constexpr size_t pad32(size_t n) { return (n + 31) & ~size_t(31); }
// element offsets of the geometry arrays (in units of the element type)
constexpr size_t kRad = pad32(kMaxNr + 1);
constexpr size_t kAng = pad32(kMaxNt + 1);
constexpr size_t oRA = 0, oRB = oRA + kRad, oRV = oRB + kRad, oIDM = oRV + kRad,
                 oIDP = oIDM + kRad, oHM = oIDP + kRad, oHP = oHM + kRad, oGRAV = oHP + kRad,
                 oAR = oGRAV + kRad, oAT = oAR + kAng, oAV = oAT + kAng, oNR = oAV + kAng,
                 oNTH = oNR + pad32(3 * (size_t)kMaxCols),
                 oNPH = oNTH + pad32(3 * ((size_t)kMaxCols + kMaxNp)),
                 oRHAT = oNPH + pad32(2 * (size_t)kMaxNp),
                 kGeoElems = oRHAT + pad32(3 * (size_t)kMaxCols);
constexpr size_t kGeoBytes = kGeoElems * sizeof(double);           // sized for FP64
constexpr size_t kPartialOff = kGeoBytes;
constexpr size_t kMiscOff = kPartialOff + (size_t)kMaxBlocks * crn::RED_STRIDE * sizeof(double);
// misc: counter (4 B) | flags (4 B) | bad cell (8 B) | stats (32 doubles)
constexpr size_t kScratchBytes = kMiscOff + 16 + 32 * sizeof(double);

}  // namespace

// The shared scratch array (about 3.6 MB).  In host code its name is only a
// host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

struct DeviceSlot {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_scratch on this device
  bool geo_valid = false;
  crn_grid_desc geo_desc{};
  bool captured = false;  // a call on this device was recorded in a graph
};

std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

// errors go to the same per-thread message as every other entry point
int fail(int code, const std::string& msg) { return crn::report_error(code, msg.c_str()); }

int validate_static(const crn_grid_desc* d) {
  if (!d) return fail(CRN_E_ARG, "crn_grid_desc is NULL");
  if (d->n_r < 2 || d->n_r > kMaxNr) return fail(CRN_E_ARG, "n_r must be in [2, 1024]");
  if (d->n_theta < 2 || d->n_theta > kMaxNt) return fail(CRN_E_ARG, "n_theta must be in [2, 1024]");
  if (d->n_phi < 8 || d->n_phi % 8 != 0 || d->n_phi > kMaxNp)
    return fail(CRN_E_ARG, "n_phi must be a multiple of 8 in [8, 2048]");
  if ((int64_t)d->n_theta * d->n_phi > kMaxCols)
    return fail(CRN_E_ARG, "n_theta * n_phi exceeds the static limit of 32768 columns");
  if (d->precision != CRN_FP64 && d->precision != CRN_FP32_BULK)
    return fail(CRN_E_ARG, "precision must be CRN_FP64 or CRN_FP32_BULK");
  if (d->limiter < CRN_LIM_NONE || d->limiter > CRN_LIM_VANALBADA)
    return fail(CRN_E_ARG, "unknown limiter");
  if (!(std::isfinite(d->r_in) && std::isfinite(d->r_out) && d->r_in > 0.0 && d->r_out > d->r_in))
    return fail(CRN_E_ARG, "need 0 < r_in < r_out");
  if (!(std::isfinite(d->gamma) && d->gamma > 1.0)) return fail(CRN_E_ARG, "gamma must be > 1");
  if (!(std::isfinite(d->c_h) && d->c_h >= 0.0)) return fail(CRN_E_ARG, "c_h must be >= 0");
  if (!std::isfinite(d->g0)) return fail(CRN_E_ARG, "g0 must be finite");
  if (!(std::isfinite(d->lim_eps) && d->lim_eps >= 0.0)) return fail(CRN_E_ARG, "lim_eps must be >= 0");
  if (d->limiter == CRN_LIM_VANALBADA && !(d->lim_eps > 0.0))
    return fail(CRN_E_ARG, "the van Albada limiter needs lim_eps > 0 (its smooth form is 0/0 where both slopes vanish)");
  if (!std::isfinite(d->outer_rho_exp) || !std::isfinite(d->outer_br_exp))
    return fail(CRN_E_ARG, "outer exponents must be finite");
  if (!(d->rho_b > 0.0 && d->p_b > 0.0 && std::isfinite(d->rho_b) && std::isfinite(d->p_b)))
    return fail(CRN_E_ARG, "rho_b and p_b must be > 0");
  if ((d->inner_bc < CRN_INNER_LOW_E || d->inner_bc > CRN_INNER_LOW_E_WP) ||
      (d->outer_vr_mass != 0 && d->outer_vr_mass != 1) ||
      (d->outer_psi_extrap != 0 && d->outer_psi_extrap != 1) || d->reserved_ != 0)
    return fail(CRN_E_ARG, "bad boundary-law field");
  if (!std::isfinite(d->vr_star) || !std::isfinite(d->outer_bphi_exp) || !std::isfinite(d->outer_vphi_exp))
    return fail(CRN_E_ARG, "vr_star and the outer exponents must be finite");
  if (!(std::isfinite(d->psi_damp) && d->psi_damp >= 0.0)) return fail(CRN_E_ARG, "psi_damp must be >= 0");
  if (d->r_last != 0.0)
    return fail(CRN_E_ARG, "crn_residual_static takes the geometric radial faces only (r_last = 0)");
  return CRN_OK;
}

// geometry of the shell computed on the device (same exact integrals as the
// host geometry of crn_grid_create), written at the fixed offsets above
template <class T>
__global__ void static_geometry_kernel(T* geo, int nr, int nt, int np, double r_in, double r_out,
                                       double g0) {
  const double kPi = 3.14159265358979323846;
  const double dth = kPi / nt, dph = 2.0 * kPi / np, s2 = 2.0 * sin(0.5 * dph);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto rf = [&](int k) {
    if (k <= 0) return r_in;
    if (k >= nr) return r_out;
    return r_in * pow(r_out / r_in, (double)k / nr);
  };
  auto rc = [&](int k) {
    if (k < 0) return 2.0 * r_in - 0.5 * (rf(0) + rf(1));
    if (k >= nr) return 2.0 * r_out - 0.5 * (rf(nr - 1) + rf(nr));
    return 0.5 * (rf(k) + rf(k + 1));
  };
  for (int64_t q = t0; q <= nr; q += stride) {
    const int k = (int)q;
    const double r = rf(k);
    geo[oRA + k] = (T)(r * r);
    if (k < nr) {
      const double r1 = rf(k), r2 = rf(k + 1), c = rc(k);
      geo[oRB + k] = (T)(0.5 * (r2 - r1) * (r2 + r1));
      geo[oRV + k] = (T)((r2 - r1) * (r2 * r2 + r2 * r1 + r1 * r1) / 3.0);
      geo[oIDM + k] = (T)(1.0 / (c - rc(k - 1)));
      geo[oIDP + k] = (T)(1.0 / (rc(k + 1) - c));
      geo[oHM + k] = (T)(c - r1);
      geo[oHP + k] = (T)(r2 - c);
      geo[oGRAV + k] = (T)(g0 / (c * c));
    }
  }
  for (int64_t q = t0; q <= nt; q += stride) {
    const int j = (int)q;
    if (j < nt) {
      const double t1 = j * dth, t2 = (j + 1) * dth, tc = (j + 0.5) * dth;
      const double X = 0.5 * (dth - cos(t1 + t2) * sin(dth));
      const double Z = 0.5 * sin(t1 + t2) * sin(dth);
      geo[oAR + j] = (T)sqrt(X * X * s2 * s2 + Z * Z * dph * dph);
      geo[oAV + j] = (T)(2.0 * sin(tc) * sin(0.5 * dth) * dph);
    }
    double at = 0.0;
    if (j > 0 && j < nt) {
      const double t = j * dth, st = sin(t), ct = cos(t);
      at = st * sqrt(ct * ct * s2 * s2 + st * st * dph * dph);
    }
    geo[oAT + j] = (T)at;
  }
  const int64_t cs = (int64_t)nt * np, ts = (int64_t)(nt + 1) * np;
  for (int64_t q = t0; q < ts; q += stride) {
    const int j = (int)(q / np), i = (int)(q % np);
    const double pc = (i + 0.5) * dph;
    if (j < nt) {
      const double t1 = j * dth, t2 = (j + 1) * dth, tc = (j + 0.5) * dth;
      const double X = 0.5 * (dth - cos(t1 + t2) * sin(dth));
      const double Z = 0.5 * sin(t1 + t2) * sin(dth);
      const double a = sqrt(X * X * s2 * s2 + Z * Z * dph * dph);
      geo[oNR + q] = (T)(X * s2 * cos(pc) / a);
      geo[oNR + cs + q] = (T)(X * s2 * sin(pc) / a);
      geo[oNR + 2 * cs + q] = (T)(Z * dph / a);
      geo[oRHAT + q] = (T)(sin(tc) * cos(pc));
      geo[oRHAT + cs + q] = (T)(sin(tc) * sin(pc));
      geo[oRHAT + 2 * cs + q] = (T)cos(tc);
    }
    double nx = 0.0, ny = 0.0, nz = 0.0;
    if (j > 0 && j < nt) {
      const double t = j * dth, st = sin(t), ct = cos(t);
      const double a = st * sqrt(ct * ct * s2 * s2 + st * st * dph * dph);
      nx = st * ct * s2 * cos(pc) / a;
      ny = st * ct * s2 * sin(pc) / a;
      nz = -st * st * dph / a;
    }
    geo[oNTH + q] = (T)nx;
    geo[oNTH + ts + q] = (T)ny;
    geo[oNTH + 2 * ts + q] = (T)nz;
  }
  for (int64_t q = t0; q < np; q += stride) {
    const double p = q * dph;
    geo[oNPH + q] = (T)(-sin(p));
    geo[oNPH + np + q] = (T)cos(p);
  }
}

template <class T>
crn::Geo<T> carve(unsigned char* base, const crn_grid_desc& d) {
  T* g = reinterpret_cast<T*>(base);
  crn::Geo<T> geo;
  geo.ra = g + oRA; geo.rb = g + oRB; geo.rv = g + oRV; geo.inv_dm = g + oIDM;
  geo.inv_dp = g + oIDP; geo.hm = g + oHM; geo.hp = g + oHP; geo.grav = g + oGRAV;
  geo.ar = g + oAR; geo.at = g + oAT; geo.av = g + oAV; geo.nr = g + oNR; geo.nth = g + oNTH;
  geo.nph = g + oNPH; geo.rhat = g + oRHAT;
  geo.dtheta = (T)(3.14159265358979323846 / d.n_theta);
  return geo;
}

template <class T>
crn::Phys<T> phys_static(const crn_grid_desc& d) {
  // outer-ghost factors (r_I / r_G)^a, (r_I / r_G)^b from the last two radial faces
  const double rl = d.r_in * std::pow(d.r_out / d.r_in, (double)(d.n_r - 1) / d.n_r);
  const double rI = 0.5 * (rl + d.r_out), rG = 2.0 * d.r_out - rI;
  crn::Phys<T> ph;
  ph.gamma = (T)d.gamma;
  ph.gm1 = (T)(d.gamma - 1.0);
  ph.igm1 = (T)(1.0 / (d.gamma - 1.0));
  ph.ch = (T)d.c_h;
  ph.ch2 = (T)(d.c_h * d.c_h);
  ph.eps = (T)d.lim_eps;
  ph.rho_b = (T)d.rho_b;
  ph.p_b = (T)d.p_b;
  ph.fa = (T)std::pow(rI / rG, d.outer_rho_exp);
  ph.fb = (T)std::pow(rI / rG, d.outer_br_exp);
  ph.fbp = (T)std::pow(rI / rG, d.outer_bphi_exp);
  ph.fvr = d.outer_vr_mass ? (T)std::pow(rI / rG, 2.0 - d.outer_rho_exp) : (T)1;
  ph.fvp = (T)std::pow(rI / rG, d.outer_vphi_exp);
  ph.psi_out = d.outer_psi_extrap ? (T)1 : (T)-1;
  ph.psi_damp = (T)d.psi_damp;
  ph.inner_bc = d.inner_bc;
  ph.vr_star = d.vr_star;
  return ph;
}

template <class T> struct StaticTile;
template <> struct StaticTile<double> { static constexpr int TT = 8, TP = 32; };
template <> struct StaticTile<float> { static constexpr int TT = 8, TP = 32; };

template <class T>
cudaError_t opt_in_smem() {
  constexpr int TT = StaticTile<T>::TT, TP = StaticTile<T>::TP;
  const int smem = (int)crn::TileDims<TT, TP>::template smem_bytes<T>();
  cudaError_t e = cudaFuncSetAttribute(crn::residual_tiled<T, 0, TT, TP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(crn::residual_tiled<T, 1, TT, TP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(crn::residual_tiled<T, 2, TT, TP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

bool same_geometry(const crn_grid_desc& a, const crn_grid_desc& b) {
  return a.n_r == b.n_r && a.n_theta == b.n_theta && a.n_phi == b.n_phi &&
         a.precision == b.precision && a.r_in == b.r_in && a.r_out == b.r_out && a.g0 == b.g0;
}

template <class T>
int run(const crn_grid_desc& d, unsigned char* base, const double* Br, const void* U, void* R,
        double* norms, double* dtmin, cudaStream_t st) {
  constexpr int TT = StaticTile<T>::TT, TP = StaticTile<T>::TP;
  crn::Shape sh;
  sh.nr = d.n_r;
  sh.nt = d.n_theta;
  sh.np = d.n_phi;
  sh.ncell = (int64_t)d.n_r * d.n_theta * d.n_phi;
  const int ntiles = ((sh.nt + TT - 1) / TT) * ((sh.np + TP - 1) / TP);
  int nsm = 0, per_sm = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crn::residual_tiled<T, 2, TT, TP>, TT * TP,
                                                crn::TileDims<TT, TP>::template smem_bytes<T>());
  int kc = crn::choose_kchunk(sh.nr, ntiles, (long long)std::max(nsm, 1) * std::max(per_sm, 1));
  while ((int64_t)ntiles * ((sh.nr + kc - 1) / kc) > kMaxBlocks) kc *= 2;
  const int nch = (sh.nr + kc - 1) / kc;
  crn::Reduce red;
  red.partials = reinterpret_cast<double*>(base + kPartialOff);
  red.counter = reinterpret_cast<unsigned int*>(base + kMiscOff);
  red.err_flags = reinterpret_cast<unsigned int*>(base + kMiscOff + 4);
  red.err_cell = reinterpret_cast<unsigned long long*>(base + kMiscOff + 8);
  red.norms_out = reinterpret_cast<double*>(base + kMiscOff + 16);
  red.dt_out = red.norms_out + 9;
  red.norms_user = norms;
  red.dt_user = dtmin;
  red.log_out = nullptr;
  // the arrival counter and the error word must start cleared
  cudaError_t e = cudaMemsetAsync(base + kMiscOff, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kMiscOff + 8, 0xff, 8, st);
  if (e != cudaSuccess) return fail(CRN_E_CUDA, std::string("clearing the scratch: ") + cudaGetErrorString(e));
  const crn::Geo<T> geo = carve<T>(base, d);
  const crn::Phys<T> ph = phys_static<T>(d);
  const size_t smem = crn::TileDims<TT, TP>::template smem_bytes<T>();
  dim3 grid((unsigned)ntiles, (unsigned)nch);
  const T* u = static_cast<const T*>(U);
  T* r = static_cast<T*>(R);
  switch (d.limiter) {
    case CRN_LIM_NONE:
      crn::residual_tiled<T, 0, TT, TP><<<grid, TT * TP, smem, st>>>(sh, geo, ph, Br, u, r, red, kc);
      break;
    case CRN_LIM_MINMOD:
      crn::residual_tiled<T, 1, TT, TP><<<grid, TT * TP, smem, st>>>(sh, geo, ph, Br, u, r, red, kc);
      break;
    default:
      crn::residual_tiled<T, 2, TT, TP><<<grid, TT * TP, smem, st>>>(sh, geo, ph, Br, u, r, red, kc);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CRN_E_CUDA, std::string("residual launch: ") + cudaGetErrorString(e));
  return CRN_OK;
}

}  // namespace

extern "C" int crn_residual_static(const crn_grid_desc* d, const double* Br_dev, const void* U_dev,
                                   void* R_dev, double* norms9_dev, double* dtmin_dev, void* stream) {
  int rc = validate_static(d);
  if (rc != CRN_OK) return rc;
  if (!Br_dev || !U_dev || !R_dev) return fail(CRN_E_ARG, "Br_dev, U_dev and R_dev must not be NULL");
  const size_t bytes = (size_t)9 * d->n_r * d->n_theta * d->n_phi * (d->precision == CRN_FP64 ? 8 : 4);
  const char* a = static_cast<const char*>(U_dev);
  const char* b = static_cast<const char*>(R_dev);
  if (a < b + bytes && b < a + bytes) return fail(CRN_E_ARG, "U_dev and R_dev overlap");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CRN_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CRN_E_ARG, "device index out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSlot& slot = g_slots[dev];
  if (!slot.ready) {  // once per device, with that device current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      return fail(CRN_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    e = opt_in_smem<double>();
    if (e == cudaSuccess) e = opt_in_smem<float>();
    if (e != cudaSuccess) return fail(CRN_E_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    slot.base = static_cast<unsigned char*>(p);
    slot.ready = true;
  }
  // A call recorded into a graph records its own geometry build, so that a
  // replay does not depend on calls made after the capture.  Since any replay
  // may then rebuild the array with its own geometry, every uncaptured call
  // on a device where a call was captured rebuilds the geometry too.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return fail(CRN_E_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (capturing) slot.captured = true;
  if (slot.captured || !slot.geo_valid || !same_geometry(slot.geo_desc, *d)) {
    const int64_t work = (int64_t)(d->n_theta + 1) * d->n_phi;
    const unsigned nb = (unsigned)std::min<int64_t>((work + 255) / 256, 1024);
    if (d->precision == CRN_FP64)
      static_geometry_kernel<double><<<nb, 256, 0, st>>>(reinterpret_cast<double*>(slot.base), d->n_r,
                                                         d->n_theta, d->n_phi, d->r_in, d->r_out, d->g0);
    else
      static_geometry_kernel<float><<<nb, 256, 0, st>>>(reinterpret_cast<float*>(slot.base), d->n_r,
                                                        d->n_theta, d->n_phi, d->r_in, d->r_out, d->g0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CRN_E_CUDA, std::string("geometry launch: ") + cudaGetErrorString(e));
    slot.geo_desc = *d;
    slot.geo_valid = !slot.captured;
  }
  if (d->precision == CRN_FP64)
    return run<double>(*d, slot.base, Br_dev, U_dev, R_dev, norms9_dev, dtmin_dev, st);
  return run<float>(*d, slot.base, Br_dev, U_dev, R_dev, norms9_dev, dtmin_dev, st);
}
