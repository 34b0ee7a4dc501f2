// erpp_tiles.cu -- FP32 tile kernels: the kernel gather and the regularised
// source scatter (Sec. 2.4, Eq. ns_regularized_filtered; the heat kernel of
// App. A.1 factored per axis).
//
// One thread block owns one tile interior and keeps it in shared memory
// (three FP32 components, x fastest, row pitch px, plane pitch pxy).  It walks
// the tile's entries (particle pieces clipped to the tile, from the binning)
// with one warp per entry.  Lanes map to (x slot, row): lane = ix + xs * q,
// rows = (y, z) pairs of the clipped window, R = 32 / xs rows per pass; the
// pitches are chosen on the host so that the R rows of one pass hit distinct
// banks.  Each lane evaluates its x weight once and one exponential per row:
//   w(j) = 2^(-beta_x d_x^2) * 2^(-(beta_y d_y^2 + beta_z d_z^2)),
// d in grid units measured from the particle, beta = log2(e) dx^2/(2 sigma^2).
//
// Gather: per-entry partial sums of w u are reduced across the warp and added
// to the particle's accumulator in global memory (one piece per tile; most
// particles have one to three pieces).  Normalisation is applied afterwards.
// Scatter: w * f is added into the shared tile with shared-memory atomics
// (optionally with a two-sum compensation word per node); the tile is then
// written to HBM once with coalesced stores, zeros included.
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

struct Piece {
  int p;          // particle index
  int len[3];     // clipped window length per axis
  int l0[3];      // first local node (inside the tile)
  float d0[3];    // distance (grid units) of the first clipped node
};

__device__ __forceinline__ void tile_origin(const erpp_kparams& kp, int tile, int b[3],
                                            int ext[3]) {
  int txy = kp.nt[0] * kp.nt[1];
  int tz = tile / txy;
  int r = tile - tz * txy;
  int ty = r / kp.nt[0];
  int tx = r - ty * kp.nt[0];
  b[0] = tx * kp.T[0];
  b[1] = ty * kp.T[1];
  b[2] = tz * kp.T[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) ext[a] = min(b[a] + kp.T[a], kp.n[a]) - b[a];
}

__device__ __forceinline__ void decode_piece(const erpp_kparams& kp, uint32_t word,
                                             const float4* __restrict__ geo_t,
                                             const int4* __restrict__ geo_c, const int b[3],
                                             const int ext[3], Piece& pc) {
  pc.p = (int)(word & ERPP_ENTRY_PMASK);
  int code = (int)(word >> ERPP_ENTRY_PBITS);
  int m[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
  float4 gt = __ldg(&geo_t[pc.p]);
  int4 gc = __ldg(&geo_c[pc.p]);
  float t[3] = {gt.x, gt.y, gt.z};
  int c[3] = {gc.x, gc.y, gc.z};
  uint32_t pack = (uint32_t)gc.w;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int jlo = c[a] + erpp_geo_off(pack, a);
    int jhi = jlo + erpp_geo_nw(pack, a) - 1;
    int sh = m[a] * kp.n[a];
    int lo = max(jlo, b[a] + sh);
    int hi = min(jhi, b[a] + ext[a] - 1 + sh);
    pc.len[a] = hi - lo + 1;
    pc.l0[a] = lo - sh - b[a];
    pc.d0[a] = (float)(lo - c[a]) - t[a];
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_gather_f32(
    erpp_kparams kp, const float* __restrict__ u, const int32_t* __restrict__ start,
    const uint32_t* __restrict__ entries, int64_t ecap, const float4* __restrict__ geo_t,
    const int4* __restrict__ geo_c, float* __restrict__ up_acc, int64_t acc_stride) {
  extern __shared__ float smem[];
  const int tile = blockIdx.x;
  const int e0 = start[tile];
  const int e1 = (int)min((int64_t)start[tile + 1], ecap);
  if (e0 >= e1) return;
  int b[3], ext[3];
  tile_origin(kp, tile, b, ext);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  // stage the tile interior of the three components (coalesced rows)
  const int nrow = 3 * ext[1] * ext[2];
  for (int r = warp; r < nrow; r += nwarps) {
    int comp = r / (ext[1] * ext[2]);
    int yz = r - comp * ext[1] * ext[2];
    int z = yz / ext[1];
    int y = yz - z * ext[1];
    const float* src = u + comp * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0] + b[0];
    float* dst = smem + comp * kp.plane + z * kp.pxy + y * kp.px;
    for (int xx = lane; xx < ext[0]; xx += 32) dst[xx] = __ldg(src + xx);
  }
  __syncthreads();
  const int ix = lane % kp.xs, q = lane / kp.xs;
  const bool lane_on = q < kp.rows;
  for (int e = e0 + warp; e < e1; e += nwarps) {
    Piece pc;
    decode_piece(kp, __ldg(&entries[e]), geo_t, geo_c, b, ext, pc);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    const bool xon = lane_on && ix < pc.len[0];
    if (xon) {
      float dxk = pc.d0[0] + (float)ix;
      float ex = exp2f(-kp.beta[0] * dxk * dxk);
      const int nr = pc.len[1] * pc.len[2];
      int ky = q % pc.len[1], kz = q / pc.len[1];
      const float* base = smem + pc.l0[2] * kp.pxy + pc.l0[1] * kp.px + pc.l0[0] + ix;
      for (int r = q; r < nr; r += kp.rows) {
        float dy = pc.d0[1] + (float)ky, dz = pc.d0[2] + (float)kz;
        float w = ex * exp2f(-(kp.beta[1] * dy * dy + kp.beta[2] * dz * dz));
        const float* s = base + kz * kp.pxy + ky * kp.px;
        a0 = fmaf(w, s[0], a0);
        a1 = fmaf(w, s[kp.plane], a1);
        a2 = fmaf(w, s[2 * kp.plane], a2);
        ky += kp.rows;
        while (ky >= pc.len[1]) {
          ky -= pc.len[1];
          ++kz;
        }
      }
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
      atomicAdd(up_acc + pc.p, a0);
      atomicAdd(up_acc + acc_stride + pc.p, a1);
      atomicAdd(up_acc + 2 * acc_stride + pc.p, a2);
    }
  }
}

template <bool KAHAN>
__global__ void __launch_bounds__(256) k_scatter_f32(
    erpp_kparams kp, float* __restrict__ S, const int32_t* __restrict__ start,
    const uint32_t* __restrict__ entries, int64_t ecap, const float4* __restrict__ geo_t,
    const int4* __restrict__ geo_c, const float4* __restrict__ fscat) {
  extern __shared__ float smem[];
  const int tile = blockIdx.x;
  const int e0 = start[tile];
  const int e1 = (int)min((int64_t)start[tile + 1], ecap);
  int b[3], ext[3];
  tile_origin(kp, tile, b, ext);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int total = (KAHAN ? 6 : 3) * kp.plane;
  if (e0 < e1) {
    for (int k = threadIdx.x; k < total; k += blockDim.x) smem[k] = 0.f;
    __syncthreads();
    float* comp_lo = smem + 3 * kp.plane;
    const int ix = lane % kp.xs, q = lane / kp.xs;
    const bool lane_on = q < kp.rows;
    for (int e = e0 + warp; e < e1; e += nwarps) {
      Piece pc;
      uint32_t word = __ldg(&entries[e]);
      decode_piece(kp, word, geo_t, geo_c, b, ext, pc);
      const bool xon = lane_on && ix < pc.len[0];
      if (!xon) continue;
      float4 f = __ldg(&fscat[pc.p]);
      float dxk = pc.d0[0] + (float)ix;
      float ex = exp2f(-kp.beta[0] * dxk * dxk);
      float fx = f.x * ex, fy = f.y * ex, fz = f.z * ex;
      const int nr = pc.len[1] * pc.len[2];
      int ky = q % pc.len[1], kz = q / pc.len[1];
      const int base = pc.l0[2] * kp.pxy + pc.l0[1] * kp.px + pc.l0[0] + ix;
      for (int r = q; r < nr; r += kp.rows) {
        float dy = pc.d0[1] + (float)ky, dz = pc.d0[2] + (float)kz;
        float w = exp2f(-(kp.beta[1] * dy * dy + kp.beta[2] * dz * dz));
        const int idx = base + kz * kp.pxy + ky * kp.px;
        float vals[3] = {fx * w, fy * w, fz * w};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float* cell = smem + c * kp.plane + idx;
          if (KAHAN) {
            float v = vals[c];
            float old = atomicAdd(cell, v);
            float s = old + v;
            float bp = s - old;
            float err = (old - (s - bp)) + (v - bp);
            atomicAdd(comp_lo + c * kp.plane + idx, err);
          } else {
            atomicAdd(cell, vals[c]);
          }
        }
        ky += kp.rows;
        while (ky >= pc.len[1]) {
          ky -= pc.len[1];
          ++kz;
        }
      }
    }
    __syncthreads();
  }
  // write the interior once (zeros for empty tiles)
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int nrow = 3 * ext[1] * ext[2];
  const bool any = e0 < e1;
  for (int r = warp; r < nrow; r += nwarps) {
    int comp = r / (ext[1] * ext[2]);
    int yz = r - comp * ext[1] * ext[2];
    int z = yz / ext[1];
    int y = yz - z * ext[1];
    float* dst = S + comp * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0] + b[0];
    const int so = comp * kp.plane + z * kp.pxy + y * kp.px;
    for (int xx = lane; xx < ext[0]; xx += 32) {
      float v = 0.f;
      if (any) {
        v = smem[so + xx];
        if (KAHAN) v += smem[3 * kp.plane + so + xx];
      }
      dst[xx] = v;
    }
  }
}

size_t tile_smem_bytes(const erpp_kparams& kp, bool kahan) {
  return sizeof(float) * (size_t)kp.plane * (kahan ? 6 : 3);
}

}  // namespace

namespace erpp {

cudaError_t launch_gather_f32(erpp_ctx* ctx, const float* u, int64_t n, cudaStream_t st) {
  (void)n;
  const erpp_kparams& kp = ctx->kp;
  size_t sm = tile_smem_bytes(kp, false);
  cudaError_t e = cudaFuncSetAttribute(k_gather_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  k_gather_f32<<<kp.ntiles, 256, sm, st>>>(kp, u, ctx->tile_start, ctx->entries,
                                           ctx->entries_cap, ctx->geo_t, ctx->geo_c,
                                           ctx->up_acc, ctx->cap);
  return cudaGetLastError();
}

cudaError_t launch_scatter_f32(erpp_ctx* ctx, float* S, cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  bool kahan = kp.kahan != 0;
  size_t sm = tile_smem_bytes(kp, kahan);
  cudaError_t e;
  if (kahan) {
    e = cudaFuncSetAttribute(k_scatter_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    k_scatter_f32<true><<<kp.ntiles, 256, sm, st>>>(kp, S, ctx->tile_start, ctx->entries,
                                                    ctx->entries_cap, ctx->geo_t, ctx->geo_c,
                                                    ctx->fscat);
  } else {
    e = cudaFuncSetAttribute(k_scatter_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    k_scatter_f32<false><<<kp.ntiles, 256, sm, st>>>(kp, S, ctx->tile_start, ctx->entries,
                                                     ctx->entries_cap, ctx->geo_t, ctx->geo_c,
                                                     ctx->fscat);
  }
  return cudaGetLastError();
}

}  // namespace erpp
