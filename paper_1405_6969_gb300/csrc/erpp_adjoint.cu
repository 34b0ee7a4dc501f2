// erpp_adjoint.cu -- adjoints of the regularised scatter and of the kernel
// gather with respect to particle forces and positions.
//
// With W_p(j) = prod_a w_a(j_a) the per-axis factored Gaussian of Sec. 2.4
// (App. A.1 heat kernel, truncated, optionally normalised per axis), the
// forward maps are
//   scatter  S_j   = -(1/rho_f) sum_p D_p W_p(j)          (Eq. ns_regularized_filtered)
//   gather   u_p   =  dV sum_j u_j W_p(j) + shear y_p e_x
// and for a cotangent field F (R = dL/dS, or the grid u) and a per-particle
// co-vector v (D_p, or g_p = dL/du_p) both adjoints need, per particle,
//   G_c   = sum_j F_jc W_p(j)
//   h_a   = sum_j (F_j . v_p) dW_p(j)/dx_pa,
// where the axis factor's derivative is
//   raw:         dw/dx_p = w d / sigma_R^2,           d = x_j - x_p,
//   normalised:  dw/dx_p = w (d - dx sum_k w_k d_k) / sigma_R^2
// (the second term is the derivative of the normalising sum).  Then
//   scatter backward:  dL/dD_pc = -(1/rho_f) G_c,  dL/dx_pa = -(1/rho_f) h_a
//   gather backward:   dL/dx_pa = dV h_a + [a = y] shear g_px,
// and the gather backward's grid part dL/du_j = dV sum_p g_p W_p(j) is a
// scatter of g (done by the scatter kernels with a force scale).
//
// One warp per particle: lanes evaluate the three axis windows and weights
// (one node per lane), then walk the (y, z) rows of the window, each lane a
// row, summing along x in the inner loop: per row A = sum_x F w_x and
// B = sum_x F w'_x, then G += A w_y w_z and h += (B w_y w_z, A w'_y w_z,
// A w_y w'_z) contracted with v.  T = float (FP32 context: weights and sums
// in FP32) or double (FP64 context).
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxW = 32;

template <typename T>
struct AxisW {
  T w[kMaxW];
  T dw[kMaxW];
};

template <typename T>
__device__ __forceinline__ T t_exp(T v);
template <>
__device__ __forceinline__ float t_exp<float>(float v) {
  return expf(v);
}
template <>
__device__ __forceinline__ double t_exp<double>(double v) {
  return exp(v);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Weights and derivative weights of one axis into aw (lane k holds node k of
// the window); returns the window length, 0 for an invalid position.
template <typename T>
__device__ int axis_weights_adj(const erpp_kparams& kp, int a, double x, AxisW<T>& aw,
                                int64_t* jlo, uint32_t* err) {
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
  const T raw1 = (T)(1.0 / sqrt(2.0 * 3.141592653589793238462643 * kp.sig2));
  const T dxa = (T)kp.dx[a];
  T wv = (T)0, d = (T)0;
  if (lane < nw) {
    d = (T)((lo + (double)lane) - s) * dxa;  // signed distance x_j - x_p
    wv = raw1 * t_exp<T>(-(d * d) / ((T)2 * sig2));
  }
  T dwv;
  if (kp.normalize) {
    const T sum = warp_sum<T>(wv);
    wv = wv / (dxa * sum);
    const T mean = dxa * warp_sum<T>(wv * d);  // dx sum_k w_k d_k
    dwv = wv * (d - mean) / sig2;
  } else {
    dwv = wv * d / sig2;
  }
  aw.w[lane] = lane < nw ? wv : (T)0;
  aw.dw[lane] = lane < nw ? dwv : (T)0;
  *jlo = (int64_t)lo;
  return nw;
}

__device__ __forceinline__ int64_t wrap_node(int64_t j, int64_t n) {
  int64_t r = j % n;
  return r < 0 ? r + n : r;
}

// outv (nullable): alpha * G; outx: alpha * h + shear_coef * v_x on the y axis.
template <typename T>
__global__ void __launch_bounds__(kWarps * 32) k_adjoint(erpp_kparams kp, int64_t n,
                                                         const double* __restrict__ x0,
                                                         const double* __restrict__ x1,
                                                         const double* __restrict__ x2,
                                                         const T* __restrict__ F,
                                                         const double* __restrict__ v0,
                                                         const double* __restrict__ v1,
                                                         const double* __restrict__ v2,
                                                         double alpha, double shear_coef,
                                                         double* ov0, double* ov1, double* ov2,
                                                         double* ox0, double* ox1, double* ox2,
                                                         uint32_t* err) {
  __shared__ AxisW<T> aw[kWarps][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t p = (int64_t)blockIdx.x * kWarps + warp;
  if (p >= n) return;
  const double xv[3] = {x0[p], x1[p], x2[p]};
  int nw[3];
  int64_t jlo[3];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nw[a] = axis_weights_adj<T>(kp, a, xv[a], aw[warp][a], &jlo[a], err);
    ok = ok && nw[a] > 0;
  }
  __syncwarp();
  const T v[3] = {(T)v0[p], (T)v1[p], (T)v2[p]};
  T G[3] = {(T)0, (T)0, (T)0};
  T h[3] = {(T)0, (T)0, (T)0};
  if (ok) {
    const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
    const AxisW<T>& wx = aw[warp][0];
    const AxisW<T>& wy = aw[warp][1];
    const AxisW<T>& wz = aw[warp][2];
    const int rows = nw[1] * nw[2];
    for (int r = lane; r < rows; r += 32) {
      const int ky = r % nw[1];
      const int kz = r / nw[1];
      const size_t rowbase =
          ((size_t)wrap_node(jlo[2] + kz, kp.n[2]) * kp.n[1] +
           (size_t)wrap_node(jlo[1] + ky, kp.n[1])) * kp.n[0];
      T A[3] = {(T)0, (T)0, (T)0}, B[3] = {(T)0, (T)0, (T)0};
      for (int kx = 0; kx < nw[0]; ++kx) {
        const size_t node = rowbase + (size_t)wrap_node(jlo[0] + kx, kp.n[0]);
        const T w = wx.w[kx], dw = wx.dw[kx];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T f = F[c * nn + node];
          A[c] += f * w;
          B[c] += f * dw;
        }
      }
      const T wyz = wy.w[ky] * wz.w[kz];
      const T dyz = wy.dw[ky] * wz.w[kz];
      const T ydz = wy.w[ky] * wz.dw[kz];
      T Av = (T)0, Bv = (T)0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        G[c] += A[c] * wyz;
        Av += A[c] * v[c];
        Bv += B[c] * v[c];
      }
      h[0] += Bv * wyz;
      h[1] += Av * dyz;
      h[2] += Av * ydz;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    G[c] = warp_sum<T>(G[c]);
    h[c] = warp_sum<T>(h[c]);
  }
  if (lane == 0) {
    if (ov0) {
      ov0[p] = alpha * (double)G[0];
      ov1[p] = alpha * (double)G[1];
      ov2[p] = alpha * (double)G[2];
    }
    ox0[p] = alpha * (double)h[0];
    ox1[p] = alpha * (double)h[1] + (ok ? shear_coef * v0[p] : 0.0);
    ox2[p] = alpha * (double)h[2];
  }
}

}  // namespace

namespace erpp {

cudaError_t launch_adjoint(erpp_ctx* ctx, int64_t n, const double* const x[3], const void* F,
                           const double* const v[3], double alpha, double shear_coef,
                           double* const outv[3], double* const outx[3], cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + kWarps - 1) / kWarps);
  double* ov[3] = {nullptr, nullptr, nullptr};
  if (outv)
    for (int a = 0; a < 3; ++a) ov[a] = outv[a];
  if (ctx->fp64) {
    k_adjoint<double><<<blocks, kWarps * 32, 0, st>>>(
        ctx->kp, n, x[0], x[1], x[2], (const double*)F, v[0], v[1], v[2], alpha, shear_coef,
        ov[0], ov[1], ov[2], outx[0], outx[1], outx[2], ctx->err);
  } else {
    k_adjoint<float><<<blocks, kWarps * 32, 0, st>>>(
        ctx->kp, n, x[0], x[1], x[2], (const float*)F, v[0], v[1], v[2], alpha, shear_coef,
        ov[0], ov[1], ov[2], outx[0], outx[1], outx[2], ctx->err);
  }
  return cudaGetLastError();
}

}  // namespace erpp
