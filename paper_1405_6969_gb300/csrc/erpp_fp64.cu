// erpp_fp64.cu -- the plain FP64 form of the gather and the scatter.
//
// One warp per particle, particles in index order, no binning: the lanes
// evaluate the per-axis weights of Sec. 2.4's truncated Gaussian in double
// precision, then walk the flattened window.  The gather reads the grid from
// global memory; the scatter adds fscale * D_p W_p(j) (fscale = -1/rho_f for
// the source) into the zeroed grid with FP64 global atomics.  This is the straightforward double-precision implementation the
// FP32 tile kernels are measured against.
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxW = 32;

// Weights of one axis (raw or normalised) into w[0..nw); returns nw (0 on an
// invalid position).
__device__ int axis_weights_f64(const erpp_kparams& kp, int a, double x, double* w, int64_t* jlo,
                                uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (!(x >= 0.0 && x < kp.L[a])) {
    if (lane == 0) erpp_set_err(err, ERPP_ERRBIT_RANGE);
    return 0;
  }
  double s, lo, hi;
  erpp_axis_window(x, kp.inv_dx[a], kp.cp[a], &s, &lo, &hi);
  int nw = (int)(hi - lo) + 1;
  if (nw > kMaxW || nw < 1) {
    if (lane == 0) erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
    return 0;
  }
  const double raw1 = 1.0 / sqrt(2.0 * 3.141592653589793238462643 * kp.sig2);
  double wv = 0.0;
  if (lane < nw) {
    double d = ((lo + (double)lane) - s) * kp.dx[a];
    wv = raw1 * exp(-(d * d) / (2.0 * kp.sig2));
  }
  if (kp.normalize) {
    double sum = wv;
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    wv = wv / (kp.dx[a] * sum);
  }
  w[lane] = wv;
  *jlo = (int64_t)lo;
  return nw;
}

__device__ __forceinline__ int64_t wrap_idx(int64_t j, int64_t n) {
  int64_t r = j % n;
  return r < 0 ? r + n : r;
}

__global__ void __launch_bounds__(kWarps * 32) k_gather_f64(erpp_kparams kp, int64_t n,
                                                            const double* __restrict__ x0,
                                                            const double* __restrict__ x1,
                                                            const double* __restrict__ x2,
                                                            const double* __restrict__ u,
                                                            double* up0, double* up1, double* up2,
                                                            uint32_t* err) {
  __shared__ double w[kWarps][3][kMaxW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t p = (int64_t)blockIdx.x * kWarps + warp;
  if (p >= n) return;
  const double xv[3] = {x0[p], x1[p], x2[p]};
  int nw[3];
  int64_t jlo[3];
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    nw[a] = axis_weights_f64(kp, a, xv[a], w[warp][a], &jlo[a], err);
    ok = ok && nw[a] > 0;
  }
  __syncwarp();
  double acc[3] = {0.0, 0.0, 0.0};
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  if (ok) {
    const int total = nw[0] * nw[1] * nw[2];
    for (int f = lane; f < total; f += 32) {
      int kx = f % nw[0];
      int t = f / nw[0];
      int ky = t % nw[1];
      int kz = t / nw[1];
      size_t node = ((size_t)wrap_idx(jlo[2] + kz, kp.n[2]) * kp.n[1] +
                     (size_t)wrap_idx(jlo[1] + ky, kp.n[1])) * kp.n[0] +
                    (size_t)wrap_idx(jlo[0] + kx, kp.n[0]);
      double W = kp.dV * (w[warp][0][kx] * w[warp][1][ky] * w[warp][2][kz]);
      acc[0] += W * u[node];
      acc[1] += W * u[nn + node];
      acc[2] += W * u[2 * nn + node];
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane == 0) {
    up0[p] = acc[0] + kp.shear_rate * xv[1];
    up1[p] = acc[1];
    up2[p] = acc[2];
  }
}

__global__ void __launch_bounds__(kWarps * 32) k_scatter_f64(erpp_kparams kp, int64_t n,
                                                             const double* __restrict__ x0,
                                                             const double* __restrict__ x1,
                                                             const double* __restrict__ x2,
                                                             const double* __restrict__ D0,
                                                             const double* __restrict__ D1,
                                                             const double* __restrict__ D2,
                                                             double fscale, double* S,
                                                             uint32_t* err) {
  __shared__ double w[kWarps][3][kMaxW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t p = (int64_t)blockIdx.x * kWarps + warp;
  if (p >= n) return;
  const double xv[3] = {x0[p], x1[p], x2[p]};
  int nw[3];
  int64_t jlo[3];
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    nw[a] = axis_weights_f64(kp, a, xv[a], w[warp][a], &jlo[a], err);
    ok = ok && nw[a] > 0;
  }
  __syncwarp();
  if (!ok) return;
  const double f[3] = {fscale * D0[p], fscale * D1[p], fscale * D2[p]};
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int total = nw[0] * nw[1] * nw[2];
  for (int fi = lane; fi < total; fi += 32) {
    int kx = fi % nw[0];
    int t = fi / nw[0];
    int ky = t % nw[1];
    int kz = t / nw[1];
    size_t node = ((size_t)wrap_idx(jlo[2] + kz, kp.n[2]) * kp.n[1] +
                   (size_t)wrap_idx(jlo[1] + ky, kp.n[1])) * kp.n[0] +
                  (size_t)wrap_idx(jlo[0] + kx, kp.n[0]);
    double W = w[warp][0][kx] * w[warp][1][ky] * w[warp][2][kz];
    atomicAdd(S + node, f[0] * W);
    atomicAdd(S + nn + node, f[1] * W);
    atomicAdd(S + 2 * nn + node, f[2] * W);
  }
}

}  // namespace

namespace erpp {

cudaError_t launch_gather_f64(erpp_ctx* ctx, const double* u, int64_t n,
                              const double* const x[3], double* const up[3], cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + kWarps - 1) / kWarps);
  ++ctx->launches;
  k_gather_f64<<<blocks, kWarps * 32, 0, st>>>(ctx->kp, n, x[0], x[1], x[2], u, up[0], up[1],
                                               up[2], ctx->err);
  return cudaGetLastError();
}

cudaError_t launch_scatter_f64(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               const double* const D[3], double fscale, double* S,
                               cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double) * 3 * nn, st);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + kWarps - 1) / kWarps);
  ++ctx->launches;
  k_scatter_f64<<<blocks, kWarps * 32, 0, st>>>(kp, n, x[0], x[1], x[2], D[0], D[1], D[2],
                                                fscale, S, ctx->err);
  return cudaGetLastError();
}

}  // namespace erpp
