// host_io.cu -- residuals of states held in host memory, with the host<->device
// copies of consecutive states overlapped with the residual kernel.
//
// Two device staging slots (U, R, norms) per grid; state i uses slot i % 2.
// The copy of U_i in runs on an input stream, the residual on the caller's
// stream, the copy of R_i out on an output stream, so that in steady state
// U_{i+1} moves in and R_{i-1} moves out while R_i is computed.  Events order
// the reuse of a slot: U_i's copy waits for the residual of state i - 2 (which
// read that slot), the residual of state i waits for the copy of R_{i-2} out.
#include <cmath>
#include <string>

#include "corona_internal.h"

namespace crn {

struct HostPipe {
  void* U[2] = {nullptr, nullptr};
  void* R[2] = {nullptr, nullptr};
  double* nrm[2] = {nullptr, nullptr};  // 9 norms + dtmin per slot
  cudaStream_t sin = nullptr, sout = nullptr;
  cudaEvent_t ein[2] = {}, ecmp[2] = {}, eout[2] = {};
  cudaEvent_t estart = nullptr, edone = nullptr;
};

void host_pipe_free(HostPipe* p) {
  if (!p) return;
  for (int s = 0; s < 2; ++s) {
    cudaFree(p->U[s]);
    cudaFree(p->R[s]);
    cudaFree(p->nrm[s]);
    if (p->ein[s]) cudaEventDestroy(p->ein[s]);
    if (p->ecmp[s]) cudaEventDestroy(p->ecmp[s]);
    if (p->eout[s]) cudaEventDestroy(p->eout[s]);
  }
  if (p->estart) cudaEventDestroy(p->estart);
  if (p->edone) cudaEventDestroy(p->edone);
  if (p->sin) cudaStreamDestroy(p->sin);
  if (p->sout) cudaStreamDestroy(p->sout);
  delete p;
}

namespace {

int report(int code, const std::string& m) { return report_error(code, m.c_str()); }

cudaError_t ensure_pipe(crn_grid* g) {
  if (g->pipe) return cudaSuccess;
  HostPipe* p = new HostPipe();
  const size_t bytes = (size_t)9 * g->shape.ncell * (g->d.precision == CRN_FP64 ? 8 : 4);
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
    e = cudaMalloc(&p->U[s], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->R[s], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->nrm[s], 10 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ein[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ecmp[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->eout[s], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->estart, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->edone, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->sin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->sout, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    host_pipe_free(p);
    return e;
  }
  g->pipe = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace crn

extern "C" {

int crn_residual_host_batch(crn_grid* g, const void* const* U_host, void* const* R_host, double* norms9_host,
                            double* dtmin_host, int32_t count, void* stream) {
  if (!g) return crn::report(CRN_E_ARG, "grid is NULL");
  if (!g->have_br) return crn::report(CRN_E_STATE, "crn_set_inner_boundary has not been called");
  if (count < 0) return crn::report(CRN_E_ARG, "count must be >= 0");
  if (count > 0 && (!U_host || !R_host)) return crn::report(CRN_E_ARG, "U_host and R_host must not be NULL");
  for (int i = 0; i < count; ++i)
    if (!U_host[i] || !R_host[i]) return crn::report(CRN_E_ARG, "state " + std::to_string(i) + ": NULL buffer");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != g->device) return crn::report(CRN_E_ARG, "the current CUDA device is not the grid's device");
  cudaError_t e = crn::ensure_pipe(g);
  if (e != cudaSuccess) return crn::report(CRN_E_CUDA, std::string("host staging: ") + cudaGetErrorString(e));
  crn::HostPipe* p = g->pipe;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)9 * g->shape.ncell * (g->d.precision == CRN_FP64 ? 8 : 4);
  int launches = 0;
  // the side streams start after the caller's earlier work
  e = cudaEventRecord(p->estart, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->sin, p->estart, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->sout, p->estart, 0);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    const int s = i & 1;
    if (i >= 2) e = cudaStreamWaitEvent(p->sin, p->ecmp[s], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->U[s], U_host[i], bytes, cudaMemcpyHostToDevice, p->sin);
    if (e == cudaSuccess) e = cudaEventRecord(p->ein[s], p->sin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ein[s], 0);
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(st, p->eout[s], 0);
    if (e != cudaSuccess) break;
    int nl = 0;
    e = g->d.precision == CRN_FP64
            ? crn::launch_residual_fp64(g, (const double*)p->U[s], (double*)p->R[s], p->nrm[s], p->nrm[s] + 9,
                                        st, &nl)
            : crn::launch_residual_fp32(g, (const float*)p->U[s], (float*)p->R[s], p->nrm[s], p->nrm[s] + 9, st,
                                        &nl);
    launches += nl;
    if (e == cudaSuccess) e = cudaEventRecord(p->ecmp[s], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->sout, p->ecmp[s], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R_host[i], p->R[s], bytes, cudaMemcpyDeviceToHost, p->sout);
    if (e == cudaSuccess && norms9_host)
      e = cudaMemcpyAsync(norms9_host + 9 * (size_t)i, p->nrm[s], 9 * sizeof(double), cudaMemcpyDeviceToHost,
                          p->sout);
    if (e == cudaSuccess && dtmin_host)
      e = cudaMemcpyAsync(dtmin_host + i, p->nrm[s] + 9, sizeof(double), cudaMemcpyDeviceToHost, p->sout);
    if (e == cudaSuccess) e = cudaEventRecord(p->eout[s], p->sout);
  }
  // join: the caller's stream waits for the last copy out; then wait on the host
  if (e == cudaSuccess) e = cudaEventRecord(p->edone, p->sout);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->edone, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  g->last_launches = launches;
  if (e != cudaSuccess) return crn::report(CRN_E_CUDA, std::string("crn_residual_host_batch: ") + cudaGetErrorString(e));
  return CRN_OK;
}

}  // extern "C"
