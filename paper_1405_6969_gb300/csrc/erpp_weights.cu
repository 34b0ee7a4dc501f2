// erpp_weights.cu -- the coupling with other weights on the same grid.
//
// ERPP_PIC: the classical particle-in-cell coupling the paper compares the
// ERPP method with (Sec. 3.2.1-3.2.2): trilinear (cloud-in-cell) weights over
// the 8 nodes of the particle's cell, for the projection of the force and the
// interpolation of the fluid velocity.
// ERPP_POINT_GATHER: the fluid velocity at the particle point by separable
// 4-point Lagrange (cubic) interpolation (the point-value reading of the
// interpolation of Sec. 2.5); the source stays the regularised kernel.
//
// Cell of a particle, per axis: s = x * (N / L) rounded once, j0 = floor(s),
// f = s - j0 (exact), node indices wrapped modulo N.
//
// The particles are first put in the order of the 8 x 8 x 8-node block of
// their cell (a counting sort: count with returning atomics, scan, fill), so
// that neighbouring lanes touch neighbouring nodes and the grid lines they
// share meet in L2 instead of being fetched from HBM per particle.  An 8-node
// PIC stencil has nothing worth staging: the PIC kernels run straight on
// global memory with two lanes per particle (one per x-neighbour), the source
// adding into the zeroed grid with device atomics (red.global.add; FP32 sums
// depend on the order of arrival).  The Lagrange gather gives each particle 4
// lanes, one per x-column of its 4 x 4 x 4 stencil, summed by shuffles, so
// that each row's 4 nodes are read by one warp instruction.  Weights are
// evaluated in the grid's type (the cell decision in FP64).
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Cell of one coordinate; false (and nothing written) outside [0, L) or NaN.
__device__ __forceinline__ bool cell_axis(const erpp_kparams& kp, int a, double x, int64_t* j0,
                                          double* f) {
  if (!(x >= 0.0 && x < kp.L[a])) return false;
  const double s = __dmul_rn(x, kp.inv_dx[a]);
  const double fl = floor(s);
  *f = s - fl;
  int64_t j = (int64_t)fl;
  if (j >= kp.n[a]) j -= kp.n[a];  // x just below L may round to s = N
  *j0 = j;
  return true;
}

__device__ __forceinline__ int64_t wrap_up(int64_t j, int64_t n) { return j >= n ? j - n : j; }
__device__ __forceinline__ int64_t wrap_down(int64_t j, int64_t n) { return j < 0 ? j + n : j; }

// Cubic Lagrange basis on the offsets -1, 0, 1, 2 at f in [0, 1).
template <typename T>
__device__ __forceinline__ void lagrange4(T f, T w[4]) {
  const T one = T(1), two = T(2);
  w[0] = -(f * (f - one) * (f - two)) / T(6);
  w[1] = ((f + one) * (f - one) * (f - two)) / two;
  w[2] = -((f + one) * f * (f - two)) / two;
  w[3] = ((f + one) * f * (f - one)) / T(6);
}

// w[k] for a lane-dependent k, by selects (no local-memory indexing).
template <typename T>
__device__ __forceinline__ T pick4(const T w[4], int k) {
  return k == 0 ? w[0] : k == 1 ? w[1] : k == 2 ? w[2] : w[3];
}

// PIC kernels: 2 lanes per particle, lane dx taking the nodes j0_x + dx, so
// that the two x-neighbours of a row go out in one warp instruction (one
// sector for both, where the row does not wrap).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_scatter_pic(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, const double* __restrict__ D0, const double* __restrict__ D1,
    const double* __restrict__ D2, double coef, const int32_t* __restrict__ perm,
    T* __restrict__ S, uint32_t* err) {
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int dx = threadIdx.x & 1;
  const int64_t stride = (int64_t)gridDim.x * (kThreads / 2);
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / 2) + (threadIdx.x >> 1); i < n;
       i += stride) {
    const int64_t p = perm[i];
    int64_t j0[3];
    double f[3];
    if (!cell_axis(kp, 0, x0[p], &j0[0], &f[0]) || !cell_axis(kp, 1, x1[p], &j0[1], &f[1]) ||
        !cell_axis(kp, 2, x2[p], &j0[2], &f[2])) {
      if (dx == 0) erpp_set_err(err, ERPP_ERRBIT_RANGE);
      continue;
    }
    // weights and products in the grid's type
    const T F[3] = {(T)(coef * D0[p]), (T)(coef * D1[p]), (T)(coef * D2[p])};
    const T fx = (T)f[0], fy = (T)f[1], fz = (T)f[2];
    const T wx = dx ? fx : T(1) - fx;
    const size_t jx = (size_t)(dx ? wrap_up(j0[0] + 1, kp.n[0]) : j0[0]);
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
      const T wz = dz ? fz : T(1) - fz;
      const size_t jz = (size_t)(dz ? wrap_up(j0[2] + 1, kp.n[2]) : j0[2]);
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const T wy = dy ? fy : T(1) - fy;
        const size_t jy = (size_t)(dy ? wrap_up(j0[1] + 1, kp.n[1]) : j0[1]);
        const T W = (wx * wy) * wz;
        const size_t node = (jz * kp.n[1] + jy) * kp.n[0] + jx;
        atomicAdd(S + node, F[0] * W);
        atomicAdd(S + nn + node, F[1] * W);
        atomicAdd(S + 2 * nn + node, F[2] * W);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_gather_pic(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, const T* __restrict__ u, const int32_t* __restrict__ perm,
    double* __restrict__ up0, double* __restrict__ up1, double* __restrict__ up2,
    uint32_t* err) {
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int dx = threadIdx.x & 1;
  const int64_t stride = (int64_t)gridDim.x * (kThreads / 2);
  // both lanes of a pair take every iteration (the shuffle below): the bound
  // rounds n up to whole warps of pairs
  const int64_t nr = (n + 15) & ~(int64_t)15;
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / 2) + (threadIdx.x >> 1); i < nr;
       i += stride) {
    const bool live = i < n;
    const int64_t p = live ? perm[i] : 0;
    double xv[3] = {0.0, 0.0, 0.0};
    int64_t j0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    bool ok = false;
    if (live) {
      xv[0] = x0[p];
      xv[1] = x1[p];
      xv[2] = x2[p];
      ok = cell_axis(kp, 0, xv[0], &j0[0], &f[0]) && cell_axis(kp, 1, xv[1], &j0[1], &f[1]) &&
           cell_axis(kp, 2, xv[2], &j0[2], &f[2]);
      if (!ok && dx == 0) erpp_set_err(err, ERPP_ERRBIT_RANGE);
    }
    T acc[3] = {T(0), T(0), T(0)};
    if (ok) {
      const T fx = (T)f[0], fy = (T)f[1], fz = (T)f[2];
      const T wx = dx ? fx : T(1) - fx;
      const size_t jx = (size_t)(dx ? wrap_up(j0[0] + 1, kp.n[0]) : j0[0]);
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const T wz = dz ? fz : T(1) - fz;
        const size_t jz = (size_t)(dz ? wrap_up(j0[2] + 1, kp.n[2]) : j0[2]);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const T wy = dy ? fy : T(1) - fy;
          const size_t jy = (size_t)(dy ? wrap_up(j0[1] + 1, kp.n[1]) : j0[1]);
          const T W = (wx * wy) * wz;
          const size_t node = (jz * kp.n[1] + jy) * kp.n[0] + jx;
          acc[0] += W * u[node];
          acc[1] += W * u[nn + node];
          acc[2] += W * u[2 * nn + node];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
    if (live && dx == 0) {
      up0[p] = (double)acc[0] + kp.shear_rate * xv[1];
      up1[p] = (double)acc[1];
      up2[p] = (double)acc[2];
    }
  }
}

// Point-value gather: 4 lanes per particle, lane kx taking the node column
// j0_x - 1 + kx of all 16 (y, z) rows of the 4 x 4 x 4 Lagrange stencil, so
// that each row's 4 nodes go out in one warp instruction.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gather_point(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, const T* __restrict__ u, const int32_t* __restrict__ perm,
    double* __restrict__ up0, double* __restrict__ up1, double* __restrict__ up2,
    uint32_t* err) {
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int kx = threadIdx.x & 3;
  const int64_t stride = (int64_t)gridDim.x * (kThreads / 4);
  // every lane of a warp runs the same number of iterations (the shuffles
  // below take the whole warp): the bound rounds n up to whole warps
  const int64_t nr = (n + 7) & ~(int64_t)7;
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / 4) + (threadIdx.x >> 2); i < nr;
       i += stride) {
    const bool live = i < n;
    const int64_t p = live ? perm[i] : 0;
    double xv[3] = {0.0, 0.0, 0.0};
    int64_t j0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    bool ok = false;
    if (live) {
      xv[0] = x0[p];
      xv[1] = x1[p];
      xv[2] = x2[p];
      ok = cell_axis(kp, 0, xv[0], &j0[0], &f[0]) && cell_axis(kp, 1, xv[1], &j0[1], &f[1]) &&
           cell_axis(kp, 2, xv[2], &j0[2], &f[2]);
      if (!ok && kx == 0) erpp_set_err(err, ERPP_ERRBIT_RANGE);
    }
    T acc[3] = {T(0), T(0), T(0)};
    if (ok) {
      T wx[4], wy[4], wz[4];
      lagrange4<T>((T)f[0], wx);
      lagrange4<T>((T)f[1], wy);
      lagrange4<T>((T)f[2], wz);
      const T wxk = pick4<T>(wx, kx);
      const size_t jx = (size_t)wrap_up(wrap_down(j0[0] - 1 + kx, kp.n[0]), kp.n[0]);
#pragma unroll
      for (int kz = 0; kz < 4; ++kz) {
        const size_t jz = (size_t)wrap_up(wrap_down(j0[2] - 1 + kz, kp.n[2]), kp.n[2]);
#pragma unroll
        for (int ky = 0; ky < 4; ++ky) {
          const size_t jy = (size_t)wrap_up(wrap_down(j0[1] - 1 + ky, kp.n[1]), kp.n[1]);
          const size_t node = (jz * kp.n[1] + jy) * kp.n[0] + jx;
          const T W = wxk * (wy[ky] * wz[kz]);
          acc[0] += W * u[node];
          acc[1] += W * u[nn + node];
          acc[2] += W * u[2 * nn + node];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      for (int o = 2; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (live && kx == 0) {
      up0[p] = (double)acc[0] + kp.shear_rate * xv[1];
      up1[p] = (double)acc[1];
      up2[p] = (double)acc[2];
    }
  }
}

// Sort key of a particle: its cell's 8 x 8 x 8-node block, x fastest; one
// extra bin (the last) for positions outside the box, which the kernels then
// report.
__global__ void __launch_bounds__(kThreads) k_block_count(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, int bx, int by, int nbins, int32_t* __restrict__ cnt,
    int32_t* __restrict__ key, int32_t* __restrict__ slot) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int64_t j0[3];
    double f[3];
    int k = nbins - 1;
    if (cell_axis(kp, 0, x0[p], &j0[0], &f[0]) && cell_axis(kp, 1, x1[p], &j0[1], &f[1]) &&
        cell_axis(kp, 2, x2[p], &j0[2], &f[2]))
      k = (int)(((j0[2] >> 3) * by + (j0[1] >> 3)) * bx + (j0[0] >> 3));
    key[p] = k;
    slot[p] = atomicAdd(cnt + k, 1);
  }
}

__global__ void __launch_bounds__(kThreads) k_block_fill(int64_t n,
                                                         const int32_t* __restrict__ key,
                                                         const int32_t* __restrict__ slot,
                                                         const int32_t* __restrict__ start,
                                                         int32_t* __restrict__ perm) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    perm[start[key[p]] + slot[p]] = (int32_t)p;
}

int blocks_for(int64_t work, int per_block) {
  int64_t b = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)152 * 16;  // grid-stride beyond 16 blocks per SM
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

namespace erpp {

cudaError_t sort_by_cell_block(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const erpp_kparams& kp = ctx->kp;
  const int bx = (kp.n[0] + 7) / 8, by = (kp.n[1] + 7) / 8;
  cudaError_t e = cudaMemsetAsync(ctx->w_cnt, 0, sizeof(int32_t) * ctx->w_nbins, st);
  if (e != cudaSuccess) return e;
  const int b = blocks_for(n, kThreads);
  ++ctx->launches;
  k_block_count<<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], bx, by, ctx->w_nbins,
                                        ctx->w_cnt, ctx->w_key, ctx->w_slot);
  e = launch_scan(ctx, ctx->w_cnt, ctx->w_start, ctx->w_tmp, ctx->w_nbins, st);
  if (e != cudaSuccess) return e;
  ++ctx->launches;
  k_block_fill<<<b, kThreads, 0, st>>>(n, ctx->w_key, ctx->w_slot, ctx->w_start, ctx->w_perm);
  return cudaGetLastError();
}

cudaError_t launch_gather_weights(erpp_ctx* ctx, const void* u, int64_t n,
                                  const double* const x[3], double* const up[3], cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const erpp_kparams& kp = ctx->kp;
  ++ctx->launches;
  if (kp.weights == ERPP_W_PIC) {
    const int b = blocks_for(n, kThreads / 2);
    if (ctx->fp64)
      k_gather_pic<double><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], (const double*)u,
                                                   ctx->w_perm, up[0], up[1], up[2], ctx->err);
    else
      k_gather_pic<float><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], (const float*)u,
                                                  ctx->w_perm, up[0], up[1], up[2], ctx->err);
  } else {
    const int b = blocks_for(n, kThreads / 4);
    if (ctx->fp64)
      k_gather_point<double><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2],
                                                     (const double*)u, ctx->w_perm, up[0],
                                                     up[1], up[2], ctx->err);
    else
      k_gather_point<float><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], (const float*)u,
                                                    ctx->w_perm, up[0], up[1], up[2], ctx->err);
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter_pic(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               const double* const D[3], double fscale, void* S,
                               cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const size_t elem = ctx->fp64 ? sizeof(double) : sizeof(float);
  cudaError_t e = cudaMemsetAsync(S, 0, elem * 3 * nn, st);
  if (e != cudaSuccess || n <= 0) return e;
  const double coef = fscale / kp.dV;
  const int b = blocks_for(n, kThreads / 2);
  ++ctx->launches;
  if (ctx->fp64)
    k_scatter_pic<double><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], D[0], D[1], D[2], coef,
                                                  ctx->w_perm, (double*)S, ctx->err);
  else
    k_scatter_pic<float><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], D[0], D[1], D[2], coef,
                                                 ctx->w_perm, (float*)S, ctx->err);
  return cudaGetLastError();
}

}  // namespace erpp
