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
// An 8-node PIC stencil has nothing to stage: the PIC kernels run one thread
// per particle straight on global memory, the scatter adding into the zeroed
// grid with device atomics (red.global.add; FP32 sums depend on the order of
// arrival).  The particles are first put in the order of the 8 x 8 x 8-node
// block of their cell (a counting sort: count with returning atomics, scan,
// fill), so that neighbouring threads touch neighbouring nodes and the grid
// lines they share meet in L2 instead of being fetched from HBM per particle.  The weights are evaluated in the grid's type (the cell decision
// in FP64).  The Lagrange gather gives each particle 16 lanes, one per
// (y, z) row of 4 x-nodes, and sums the rows by shuffles: its 64 nodes are
// read as 16 short row segments instead of 64 scattered words.
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

template <typename T>
__global__ void __launch_bounds__(kThreads) k_scatter_pic(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, const double* __restrict__ D0, const double* __restrict__ D1,
    const double* __restrict__ D2, double coef, const int32_t* __restrict__ perm,
    T* __restrict__ S, uint32_t* err) {
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[i];
    int64_t j0[3];
    double f[3];
    if (!cell_axis(kp, 0, x0[p], &j0[0], &f[0]) || !cell_axis(kp, 1, x1[p], &j0[1], &f[1]) ||
        !cell_axis(kp, 2, x2[p], &j0[2], &f[2])) {
      erpp_set_err(err, ERPP_ERRBIT_RANGE);
      continue;
    }
    // weights and products in the grid's type
    const T F[3] = {(T)(coef * D0[p]), (T)(coef * D1[p]), (T)(coef * D2[p])};
    const T fx = (T)f[0], fy = (T)f[1], fz = (T)f[2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
      const T wz = dz ? fz : T(1) - fz;
      const size_t jz = (size_t)(dz ? wrap_up(j0[2] + 1, kp.n[2]) : j0[2]);
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const T wy = dy ? fy : T(1) - fy;
        const size_t jy = (size_t)(dy ? wrap_up(j0[1] + 1, kp.n[1]) : j0[1]);
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const T wx = dx ? fx : T(1) - fx;
          const size_t jx = (size_t)(dx ? wrap_up(j0[0] + 1, kp.n[0]) : j0[0]);
          const T W = (wx * wy) * wz;
          const size_t node = (jz * kp.n[1] + jy) * kp.n[0] + jx;
          atomicAdd(S + node, F[0] * W);
          atomicAdd(S + nn + node, F[1] * W);
          atomicAdd(S + 2 * nn + node, F[2] * W);
        }
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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[i];
    const double xv[3] = {x0[p], x1[p], x2[p]};
    int64_t j0[3];
    double f[3];
    T acc[3] = {T(0), T(0), T(0)};
    if (cell_axis(kp, 0, xv[0], &j0[0], &f[0]) && cell_axis(kp, 1, xv[1], &j0[1], &f[1]) &&
        cell_axis(kp, 2, xv[2], &j0[2], &f[2])) {
      const T fx = (T)f[0], fy = (T)f[1], fz = (T)f[2];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const T wz = dz ? fz : T(1) - fz;
        const size_t jz = (size_t)(dz ? wrap_up(j0[2] + 1, kp.n[2]) : j0[2]);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const T wy = dy ? fy : T(1) - fy;
          const size_t jy = (size_t)(dy ? wrap_up(j0[1] + 1, kp.n[1]) : j0[1]);
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            const T wx = dx ? fx : T(1) - fx;
            const size_t jx = (size_t)(dx ? wrap_up(j0[0] + 1, kp.n[0]) : j0[0]);
            const T W = (wx * wy) * wz;
            const size_t node = (jz * kp.n[1] + jy) * kp.n[0] + jx;
            acc[0] += W * u[node];
            acc[1] += W * u[nn + node];
            acc[2] += W * u[2 * nn + node];
          }
        }
      }
    } else {
      erpp_set_err(err, ERPP_ERRBIT_RANGE);
    }
    up0[p] = (double)acc[0] + kp.shear_rate * xv[1];
    up1[p] = (double)acc[1];
    up2[p] = (double)acc[2];
  }
}

// 16 lanes per particle: lane r of the group takes the row (ky, kz) = (r % 4,
// r / 4) of the 4 x 4 x 4 Lagrange stencil.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gather_point(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, const T* __restrict__ u, const int32_t* __restrict__ perm,
    double* __restrict__ up0, double* __restrict__ up1, double* __restrict__ up2,
    uint32_t* err) {
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int r = threadIdx.x & 15;
  const int64_t groups = (int64_t)gridDim.x * (kThreads / 16);
  // every lane of a warp runs the same number of iterations (the shuffles
  // below take the whole warp): the loop bound rounds n up to pairs
  const int64_t n2 = (n + 1) & ~(int64_t)1;
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / 16) + (threadIdx.x >> 4); i < n2;
       i += groups) {
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
      if (!ok && r == 0) erpp_set_err(err, ERPP_ERRBIT_RANGE);
    }
    T acc[3] = {T(0), T(0), T(0)};
    if (ok) {
      T wx[4], wy[4], wz[4];
      lagrange4<T>((T)f[0], wx);
      lagrange4<T>((T)f[1], wy);
      lagrange4<T>((T)f[2], wz);
      const int ky = r & 3, kz = r >> 2;
      const size_t jz = (size_t)wrap_up(wrap_down(j0[2] - 1 + kz, kp.n[2]), kp.n[2]);
      const size_t jy = (size_t)wrap_up(wrap_down(j0[1] - 1 + ky, kp.n[1]), kp.n[1]);
      const size_t row = (jz * kp.n[1] + jy) * kp.n[0];
      const T wyz = pick4<T>(wy, ky) * pick4<T>(wz, kz);
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) {
        const size_t node = row + (size_t)wrap_up(wrap_down(j0[0] - 1 + kx, kp.n[0]), kp.n[0]);
        const T W = wx[kx] * wyz;
        acc[0] += W * u[node];
        acc[1] += W * u[nn + node];
        acc[2] += W * u[2 * nn + node];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      for (int o = 8; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (live && r == 0) {
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
    const int b = blocks_for(n, kThreads);
    if (ctx->fp64)
      k_gather_pic<double><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], (const double*)u,
                                                   ctx->w_perm, up[0], up[1], up[2], ctx->err);
    else
      k_gather_pic<float><<<b, kThreads, 0, st>>>(kp, n, x[0], x[1], x[2], (const float*)u,
                                                  ctx->w_perm, up[0], up[1], up[2], ctx->err);
  } else {
    const int b = blocks_for(n, kThreads / 16);
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
  const int b = blocks_for(n, kThreads);
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
