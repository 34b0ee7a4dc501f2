// erpp_host.cu -- the coupling step on host-resident data, pipelined.
//
// erpp_step_host takes the fluid field, the particle state and the source in
// host memory (page-locked, for the copies to be asynchronous).  Each call
// copies its inputs in (after the caller's stream's prior work), runs the
// step and copies the results out on streams of its own, with device staging
// in two slots used by alternate calls, and returns once all is enqueued;
// erpp_step_host_wait makes a stream wait for every call so far.  Successive
// calls overlap: a call's field upload runs while the
// previous call computes, and a call's source download while the next one
// computes.  The particle state travels host -> device -> host every call;
// the next call's particle upload waits for this call's particle download
// (the host arrays are the state of record), which starts as soon as the
// particles are advanced, before the scatter.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include "erpp_internal.cuh"

namespace {

constexpr int kPartArrays = 14;  // x, v, x_prev, D (3 each), radius, rho_p

}  // namespace

struct erpp_host_pipe {
  int64_t cap;           // particles per slot
  size_t grid_bytes;     // one grid (three components)
  void* u[2];
  void* S[2];
  double* p[2][kPartArrays];
  cudaStream_t s_in, s_comp, s_pout, s_sout;
  cudaEvent_t ev_caller, ev_in[2], ev_adv[2], ev_comp[2], ev_pout[2], ev_sout[2];
  int used[2];           // the slot has run a step (its events are recorded)
  int64_t calls;
};

namespace erpp {

void free_host_pipe(erpp_ctx* c) {
  erpp_host_pipe* h = c->hp;
  if (!h) return;
  cudaDeviceSynchronize();
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->u[b]);
    cudaFree(h->S[b]);
    for (int k = 0; k < kPartArrays; ++k) cudaFree(h->p[b][k]);
    cudaEventDestroy(h->ev_in[b]);
    cudaEventDestroy(h->ev_adv[b]);
    cudaEventDestroy(h->ev_comp[b]);
    cudaEventDestroy(h->ev_pout[b]);
    cudaEventDestroy(h->ev_sout[b]);
  }
  cudaEventDestroy(h->ev_caller);
  cudaStreamDestroy(h->s_in);
  cudaStreamDestroy(h->s_comp);
  cudaStreamDestroy(h->s_pout);
  cudaStreamDestroy(h->s_sout);
  free(h);
  c->hp = nullptr;
}

}  // namespace erpp

namespace {

// Pipeline with room for n particles (created or grown; growing synchronises).
erpp_status host_pipe(erpp_ctx* c, int64_t n, erpp_host_pipe** out) {
  const size_t nn = (size_t)c->kp.n[0] * c->kp.n[1] * c->kp.n[2];
  const size_t gb = 3 * nn * (c->fp64 ? sizeof(double) : sizeof(float));
  if (c->hp && c->hp->cap >= n && c->hp->grid_bytes == gb) {
    *out = c->hp;
    return ERPP_OK;
  }
  erpp::free_host_pipe(c);
  erpp_host_pipe* h = (erpp_host_pipe*)calloc(1, sizeof(erpp_host_pipe));
  if (!h) return ERPP_ENOMEM;
  c->hp = h;
  h->cap = n > 1024 ? n : 1024;
  h->grid_bytes = gb;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&h->u[b], gb);
    if (e == cudaSuccess) e = cudaMalloc(&h->S[b], gb);
    for (int k = 0; k < kPartArrays && e == cudaSuccess; ++k)
      e = cudaMalloc(&h->p[b][k], sizeof(double) * (size_t)h->cap);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_adv[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pout[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sout[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_caller, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_pout, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_sout, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    erpp::free_host_pipe(c);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? ERPP_ENOMEM : ERPP_ECUDA;
  }
  *out = h;
  return ERPP_OK;
}

}  // namespace

extern "C" {

erpp_status erpp_step_host(erpp_ctx* c, const void* u, const erpp_particles* P, void* S,
                           int first_step, erpp_stream stream) {
  if (!c || !u || !P || !S || P->n < 0 || P->n > ERPP_MAX_PARTICLES) return ERPP_EINVAL;
  const int64_t n = P->n;
  if (n > 0) {
    if (!P->radius || !P->rho_p) return ERPP_EINVAL;
    for (int a = 0; a < 3; ++a)
      if (!P->x[a] || !P->v[a] || !P->x_prev[a] || !P->D[a]) return ERPP_EINVAL;
  }
  erpp_host_pipe* h = nullptr;
  erpp_status s = host_pipe(c, n, &h);
  if (s != ERPP_OK) return s;
  const int b = (int)(h->calls & 1);
  const size_t pb = sizeof(double) * (size_t)n;
  // host arrays of the state: x, v, x_prev, D (written back), radius, rho_p
  double* hp[kPartArrays];
  for (int a = 0; a < 3; ++a) {
    hp[a] = P->x[a];
    hp[3 + a] = P->v[a];
    hp[6 + a] = P->x_prev[a];
    hp[9 + a] = P->D[a];
  }
  hp[12] = const_cast<double*>(P->radius);
  hp[13] = const_cast<double*>(P->rho_p);
  cudaStream_t caller = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(h->ev_caller, caller);  // after the caller's prior work
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_in, h->ev_caller, 0);
  // inputs: the slot's previous step must be done with its buffers
  if (e == cudaSuccess && h->used[b]) e = cudaStreamWaitEvent(h->s_in, h->ev_comp[b], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->u[b], u, h->grid_bytes, cudaMemcpyHostToDevice, h->s_in);
  // the particle arrays once the previous call has written them back
  if (e == cudaSuccess && h->used[1 - b])
    e = cudaStreamWaitEvent(h->s_in, h->ev_pout[1 - b], 0);
  for (int k = 0; k < kPartArrays && e == cudaSuccess && n > 0; ++k)
    e = cudaMemcpyAsync(h->p[b][k], hp[k], pb, cudaMemcpyHostToDevice, h->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[b], h->s_in);
  // the step, once the inputs are in and the slot's previous source is out
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_comp, h->ev_in[b], 0);
  if (e == cudaSuccess && h->used[b]) e = cudaStreamWaitEvent(h->s_comp, h->ev_sout[b], 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ERPP_ECUDA;
  }
  erpp_particles dp;
  dp.n = n;
  for (int a = 0; a < 3; ++a) {
    dp.x[a] = h->p[b][a];
    dp.v[a] = h->p[b][3 + a];
    dp.x_prev[a] = h->p[b][6 + a];
    dp.D[a] = h->p[b][9 + a];
  }
  dp.radius = h->p[b][12];
  dp.rho_p = h->p[b][13];
  s = erpp::step_device(c, h->u[b], &dp, h->S[b], first_step, h->s_comp, h->ev_adv[b]);
  if (s != ERPP_OK) return s;
  e = cudaEventRecord(h->ev_comp[b], h->s_comp);
  // results: the particle state as soon as it is advanced, the source after
  // the scatter, each on its own stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_pout, h->ev_adv[b], 0);
  for (int k = 0; k < 12 && e == cudaSuccess && n > 0; ++k)
    e = cudaMemcpyAsync(hp[k], h->p[b][k], pb, cudaMemcpyDeviceToHost, h->s_pout);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_pout[b], h->s_pout);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_sout, h->ev_comp[b], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S, h->S[b], h->grid_bytes, cudaMemcpyDeviceToHost, h->s_sout);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_sout[b], h->s_sout);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ERPP_ECUDA;
  }
  h->used[b] = 1;
  ++h->calls;
  return ERPP_OK;
}

erpp_status erpp_step_host_wait(erpp_ctx* c, erpp_stream stream) {
  if (!c) return ERPP_EINVAL;
  erpp_host_pipe* h = c->hp;
  if (!h) return ERPP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    if (!h->used[b]) continue;
    e = cudaStreamWaitEvent(st, h->ev_pout[b], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_sout[b], 0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ERPP_ECUDA;
  }
  return ERPP_OK;
}

}  // extern "C"
