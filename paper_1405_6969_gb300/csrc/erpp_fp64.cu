// erpp_fp64.cu -- the plain FP64 form of the gather and the scatter, and the
// gather of the velocity with its Laplacian for the general force.
//
// One warp per particle, particles in index order, no binning: the lanes
// evaluate the per-axis weights of Sec. 2.4's truncated Gaussian in double
// precision, then walk the flattened window.  The gather reads the grid from
// global memory; the scatter adds fscale * D_p W_p(j) (fscale = -1/rho_f for
// the source) into the zeroed grid with FP64 global atomics.  This is the
// straightforward double-precision implementation the FP32 tile kernels are
// measured against.
//
// The Laplacian gather (ERPP_FULL_FORCE, Eq. force_particle) walks the same
// window with the weights' second derivatives as well; on FP32 grids its
// windows are computed once per particle and its particles visited in
// cell-block order.
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

// Weights of one axis and their second derivatives in the particle
// coordinate (raw or normalised like axis_weights_f64), evaluated in FP64 and
// stored as T.  With d = (j - s) dx: dw/dx_p = w d / sig2,
// d2w/dx_p2 = w (d^2 / sig2^2 - 1 / sig2); for the normalised w~ = w / Z the
// quotient rule gives w~'' = w~ (B - 2 A m1 - m2 + 2 m1^2), A = d / sig2,
// B = d^2 / sig2^2 - 1 / sig2, m1 and m2 the w~-means of A and B.
// The window is decided in FP64 (the oracle's exact membership); the weights
// are evaluated in T from the FP64 offset of each node (FP64 arithmetic runs
// at a small fraction of the FP32 rate: FP32 contexts keep it to the window).
template <typename T>
__device__ int axis_weights_d2(const erpp_kparams& kp, int a, double x, T* w, T* w2, int* jw,
                               uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (!(x >= 0.0 && x < kp.L[a])) {
    if (lane == 0) erpp_set_err(err, ERPP_ERRBIT_RANGE);
    return 0;
  }
  double s, lo, hi;
  erpp_axis_window(x, kp.inv_dx[a], kp.cp[a], &s, &lo, &hi);
  const int nw = (int)(hi - lo) + 1;
  if (nw > kMaxW || nw < 1) {
    if (lane == 0) erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
    return 0;
  }
  const T sig2 = (T)kp.sig2;
  const T dxa = (T)kp.dx[a];
  T wv = T(0), A = T(0), B = T(0);
  if (lane < nw) {
    const T d = (T)((lo + (double)lane) - s) * dxa;
    wv = (T)kp.raw_norm1 * exp(-(d * d) / (T(2) * sig2));
    A = d / sig2;
    B = d * d / (sig2 * sig2) - T(1) / sig2;
  }
  T w2v;
  if (kp.normalize) {
    T sum = wv;
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    wv = wv / (dxa * sum);
    T m1 = dxa * wv * A, m2 = dxa * wv * B;
    for (int o = 16; o > 0; o >>= 1) {
      m1 += __shfl_xor_sync(0xffffffffu, m1, o);
      m2 += __shfl_xor_sync(0xffffffffu, m2, o);
    }
    w2v = wv * (B - T(2) * A * m1 - m2 + T(2) * m1 * m1);
  } else {
    w2v = wv * B;
  }
  w[lane] = wv;
  w2[lane] = w2v;
  if (lane < nw) {  // wrapped node index (the window starts at most 15 nodes below 0)
    int j = (int)lo + lane;
    j = j < 0 ? j + kp.n[a] : (j >= kp.n[a] ? j - kp.n[a] : j);
    jw[lane] = j;
  }
  return nw;
}

// Gather of u and of its Laplacian in the particle position, warp per
// particle; products and sums in the grid's type.
template <typename T>
__global__ void __launch_bounds__(kWarps * 32) k_gather_faxen(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, const T* __restrict__ u, double* up0, double* up1,
    double* up2, double* lap, int64_t lap_stride, uint32_t* err) {
  __shared__ T w[kWarps][3][kMaxW];
  __shared__ T w2[kWarps][3][kMaxW];
  __shared__ int jw[kWarps][3][kMaxW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t p = (int64_t)blockIdx.x * kWarps + warp;
  if (p >= n) return;
  const double xv[3] = {x0[p], x1[p], x2[p]};
  int nw[3];
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    nw[a] = axis_weights_d2<T>(kp, a, xv[a], w[warp][a], w2[warp][a], jw[warp][a], err);
    ok = ok && nw[a] > 0;
  }
  __syncwarp();
  T acc[3] = {T(0), T(0), T(0)}, lac[3] = {T(0), T(0), T(0)};
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  if (ok) {
    const int total = nw[0] * nw[1] * nw[2];
    for (int f = lane; f < total; f += 32) {
      const int kx = f % nw[0];
      const int t = f / nw[0];
      const int ky = t % nw[1];
      const int kz = t / nw[1];
      const size_t node = ((size_t)jw[warp][2][kz] * kp.n[1] + (size_t)jw[warp][1][ky]) *
                              kp.n[0] + (size_t)jw[warp][0][kx];
      const T wx = w[warp][0][kx], wy = w[warp][1][ky], wz = w[warp][2][kz];
      const T W = wx * wy * wz;
      const T K = w2[warp][0][kx] * wy * wz + wx * w2[warp][1][ky] * wz +
                  wx * wy * w2[warp][2][kz];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T uv = u[c * nn + node];
        acc[c] += W * uv;
        lac[c] += K * uv;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      lac[c] += __shfl_xor_sync(0xffffffffu, lac[c], o);
    }
  if (lane == 0) {
    up0[p] = kp.dV * (double)acc[0] + kp.shear_rate * xv[1];
    up1[p] = kp.dV * (double)acc[1];
    up2[p] = kp.dV * (double)acc[2];
    lap[p] = kp.dV * (double)lac[0];
    lap[lap_stride + p] = kp.dV * (double)lac[1];
    lap[2 * lap_stride + p] = kp.dV * (double)lac[2];
  }
}

// FP32 grids: the FP64 windows once per particle (one thread each), so that
// the gather's lanes work in FP32 only.  win[i] = (j_lo x, y, z, packed
// lengths nw_x | nw_y << 8 | nw_z << 16, 0 when invalid), frac[i] = s - j_lo
// per axis (s = x N / L).
__global__ void __launch_bounds__(256) k_faxen_windows(erpp_kparams kp, int64_t n,
                                                       const double* __restrict__ x0,
                                                       const double* __restrict__ x1,
                                                       const double* __restrict__ x2,
                                                       int4* __restrict__ win,
                                                       float4* __restrict__ frac, uint32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xv[3] = {x0[i], x1[i], x2[i]};
  int lo[3], nw[3];
  float fr[3];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(xv[a] >= 0.0 && xv[a] < kp.L[a])) {
      ok = false;
      erpp_set_err(err, ERPP_ERRBIT_RANGE);
      lo[a] = 0;
      nw[a] = 0;
      fr[a] = 0.f;
      continue;
    }
    double s, l, h;
    erpp_axis_window(xv[a], kp.inv_dx[a], kp.cp[a], &s, &l, &h);
    lo[a] = (int)l;
    nw[a] = (int)(h - l) + 1;
    fr[a] = (float)(s - l);
    if (nw[a] > kMaxW || nw[a] < 1) {
      ok = false;
      erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
    }
  }
  win[i] = make_int4(lo[0], lo[1], lo[2], ok ? (nw[0] | (nw[1] << 8) | (nw[2] << 16)) : 0);
  frac[i] = make_float4(fr[0], fr[1], fr[2], 0.f);
}

// Weights and second derivatives of one axis from a precomputed window (FP32),
// with the same formulas as axis_weights_d2.
__device__ void axis_weights_d2_f32(const erpp_kparams& kp, int a, int lo, int nw, float r,
                                    float* w, float* w2, int* jw) {
  const int lane = threadIdx.x & 31;
  const float sig2 = (float)kp.sig2;
  const float dxa = (float)kp.dx[a];
  float wv = 0.f, A = 0.f, B = 0.f;
  if (lane < nw) {
    const float d = ((float)lane - r) * dxa;
    wv = (float)kp.raw_norm1 * expf(-(d * d) / (2.f * sig2));
    A = d / sig2;
    B = d * d / (sig2 * sig2) - 1.f / sig2;
  }
  float w2v;
  if (kp.normalize) {
    float sum = wv;
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    wv = wv / (dxa * sum);
    float m1 = dxa * wv * A, m2 = dxa * wv * B;
    for (int o = 16; o > 0; o >>= 1) {
      m1 += __shfl_xor_sync(0xffffffffu, m1, o);
      m2 += __shfl_xor_sync(0xffffffffu, m2, o);
    }
    w2v = wv * (B - 2.f * A * m1 - m2 + 2.f * m1 * m1);
  } else {
    w2v = wv * B;
  }
  w[lane] = wv;
  w2[lane] = w2v;
  if (lane < nw) {
    int j = lo + lane;
    j = j < 0 ? j + kp.n[a] : (j >= kp.n[a] ? j - kp.n[a] : j);
    jw[lane] = j;
  }
}

// Particles in the order perm (by cell block), so that neighbouring warps
// read neighbouring grid rows and share them in L2.
__global__ void __launch_bounds__(kWarps * 32) k_gather_faxen_f32(
    erpp_kparams kp, int64_t n, const double* __restrict__ x1, const int4* __restrict__ win,
    const float4* __restrict__ frac, const int32_t* __restrict__ perm,
    const float* __restrict__ u, double* up0, double* up1, double* up2, double* lap,
    int64_t lap_stride) {
  __shared__ float w[kWarps][3][kMaxW];
  __shared__ float w2[kWarps][3][kMaxW];
  __shared__ int jw[kWarps][3][kMaxW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  if (i >= n) return;
  const int64_t p = perm[i];
  const int4 wi = win[p];
  const float4 fr = frac[p];
  const int nw[3] = {wi.w & 255, (wi.w >> 8) & 255, (wi.w >> 16) & 255};
  const bool ok = wi.w != 0;
  if (ok) {
    axis_weights_d2_f32(kp, 0, wi.x, nw[0], fr.x, w[warp][0], w2[warp][0], jw[warp][0]);
    axis_weights_d2_f32(kp, 1, wi.y, nw[1], fr.y, w[warp][1], w2[warp][1], jw[warp][1]);
    axis_weights_d2_f32(kp, 2, wi.z, nw[2], fr.z, w[warp][2], w2[warp][2], jw[warp][2]);
  }
  __syncwarp();
  float acc[3] = {0.f, 0.f, 0.f}, lac[3] = {0.f, 0.f, 0.f};
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  // lanes as (kx, row): lane kx = lane % nw_x of rows lane / nw_x, + R, ...
  // (R = 32 / nw_x rows per pass); the row's (ky, kz) advance without divisions
  const int R = 32 / nw[0];
  const int kx = lane % nw[0];
  int r0 = lane / nw[0];
  if (ok && r0 < R) {
    const float wx = w[warp][0][kx], w2x = w2[warp][0][kx];
    const size_t jx = (size_t)jw[warp][0][kx];
    int ky = r0 % nw[1], kz = r0 / nw[1];
    for (; kz < nw[2];) {
      const float wy = w[warp][1][ky], wz = w[warp][2][kz];
      const float w2y = w2[warp][1][ky], w2z = w2[warp][2][kz];
      const float W = wx * (wy * wz);
      const float K = w2x * (wy * wz) + wx * (w2y * wz + wy * w2z);
      const size_t node =
          ((size_t)jw[warp][2][kz] * kp.n[1] + (size_t)jw[warp][1][ky]) * kp.n[0] + jx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float uv = u[c * nn + node];
        acc[c] += W * uv;
        lac[c] += K * uv;
      }
      ky += R;
      while (ky >= nw[1]) {
        ky -= nw[1];
        ++kz;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      lac[c] += __shfl_xor_sync(0xffffffffu, lac[c], o);
    }
  if (lane == 0) {
    up0[p] = kp.dV * (double)acc[0] + kp.shear_rate * x1[p];
    up1[p] = kp.dV * (double)acc[1];
    up2[p] = kp.dV * (double)acc[2];
    lap[p] = kp.dV * (double)lac[0];
    lap[lap_stride + p] = kp.dV * (double)lac[1];
    lap[2 * lap_stride + p] = kp.dV * (double)lac[2];
  }
}

}  // namespace

namespace erpp {

cudaError_t launch_gather_faxen(erpp_ctx* ctx, const void* u, int64_t n,
                                const double* const x[3], double* const up[3], cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + kWarps - 1) / kWarps);
  if (ctx->fp64) {
    ++ctx->launches;
    k_gather_faxen<double><<<blocks, kWarps * 32, 0, st>>>(
        ctx->kp, n, x[0], x[1], x[2], (const double*)u, up[0], up[1], up[2], ctx->ff_lap,
        ctx->cap, ctx->err);
  } else {
    // FP32 grids: the particles ordered by cell block, the windows once per
    // particle into the tile path's geometry arrays (free between steps),
    // then the FP32 gather
    cudaError_t e = sort_by_cell_block(ctx, n, x, st);
    if (e != cudaSuccess) return e;
    ctx->launches += 2;
    k_faxen_windows<<<(int)((n + 255) / 256), 256, 0, st>>>(ctx->kp, n, x[0], x[1], x[2],
                                                             ctx->geo_c, ctx->geo_t, ctx->err);
    k_gather_faxen_f32<<<blocks, kWarps * 32, 0, st>>>(ctx->kp, n, x[1], ctx->geo_c, ctx->geo_t,
                                                       ctx->w_perm, (const float*)u, up[0],
                                                       up[1], up[2], ctx->ff_lap, ctx->cap);
  }
  return cudaGetLastError();
}

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
