// erpp_tiles.cu -- FP32 tile kernels: the kernel gather and the regularised
// source scatter (Sec. 2.4, Eq. ns_regularized_filtered; the heat kernel of
// App. A.1 factored per axis).
//
// One thread block owns one tile interior and keeps it in shared memory
// (three FP32 components, x fastest, row pitch px, plane pitch pxy).  The
// tile's entries (particle stencil pieces clipped to the tile, from the
// binning) are decoded in batches of 256 -- one per thread, so the global
// loads of a batch overlap -- into piece records in shared memory.  Warps then
// take groups of 8 pieces.  For one piece the lanes map to (x slot, row):
// lane = ix + xs * q, a row being one (y, z) pair of the clipped window and
// R = 32 / xs rows running per pass; the pitches are chosen on the host so
// that the R rows of a pass fall in distinct banks.  Weights are separable:
//   w = 2^(-beta_x d_x^2) * 2^(-(beta_y d_y^2 + beta_z d_z^2)),
// d in grid units from the particle, beta = log2(e) dx^2 / (2 sigma_R^2);
// each lane evaluates its x factor once per piece and one exponential per row.
//
// Gather: a lane accumulates w*u for the 8 pieces of its group in registers;
// one transpose reduction across the warp (31 shuffles for 8 pieces x 3
// components) leaves every lane with one total, added to the particle's
// accumulator in global memory.  Normalisation is applied afterwards.
//
// Scatter: contributions are accumulated exactly in 32-bit fixed point with
// shared-memory integer atomics (order independent, hence deterministic).  The
// tile's scale is the power of two 2^30 / B, B >= the sum over its pieces of
// max|f|, which bounds every node's magnitude (unnormalised weights are <= 1),
// so no sum can overflow; each contribution is rounded once, to B 2^-31.
// With ERPP_KAHAN the scatter instead adds FP32 values with shared atomics and
// keeps the exact rounding error of every addition (two-sum on the value the
// atomic returned) in a second array.  The tile is then written to HBM once
// with coalesced stores, zeros included.
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBatch = kThreads;  // pieces decoded per batch
constexpr int kGroup = 8;         // pieces per warp group
constexpr int kDenseTile = 1024;  // pieces above which a tile accumulates in compensated FP32

struct PieceSmem {
  int p[kBatch];
  int len[kBatch];   // lx | ly << 8 | lz << 16
  int base[kBatch];  // first node of the piece in the tile (shared-memory index)
  float d[3][kBatch];
  float f[3][kBatch];  // scatter: scaled force
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

// Decode one entry into its piece record (slot j of the batch).
__device__ __forceinline__ void decode_piece(const erpp_kparams& kp, uint32_t word,
                                             const float4* __restrict__ geo_t,
                                             const int4* __restrict__ geo_c, const int b[3],
                                             const int ext[3], PieceSmem& ps, int j) {
  const int p = (int)(word & ERPP_ENTRY_PMASK);
  const int code = (int)(word >> ERPP_ENTRY_PBITS);
  const int m[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
  const float4 gt = __ldg(&geo_t[p]);
  const int4 gc = __ldg(&geo_c[p]);
  const float t[3] = {gt.x, gt.y, gt.z};
  const int c[3] = {gc.x, gc.y, gc.z};
  const uint32_t pack = (uint32_t)gc.w;
  int len[3], l0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int jlo = c[a] + erpp_geo_off(pack, a);
    int jhi = jlo + erpp_geo_nw(pack, a) - 1;
    int sh = m[a] * kp.n[a];
    int lo = max(jlo, b[a] + sh);
    int hi = min(jhi, b[a] + ext[a] - 1 + sh);
    len[a] = hi - lo + 1;
    l0[a] = lo - sh - b[a];
    ps.d[a][j] = (float)(lo - c[a]) - t[a];
  }
  ps.p[j] = p;
  ps.len[j] = len[0] | (len[1] << 8) | (len[2] << 16);
  ps.base[j] = l0[2] * kp.pxy + l0[1] * kp.px + l0[0];
}

__device__ __forceinline__ void stage_tile(const erpp_kparams& kp, const float* __restrict__ u,
                                           float* smem, const int b[3], const int ext[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int nrow = 3 * ext[1] * ext[2];
  for (int r = warp; r < nrow; r += kWarps) {
    int comp = r / (ext[1] * ext[2]);
    int yz = r - comp * ext[1] * ext[2];
    int z = yz / ext[1];
    int y = yz - z * ext[1];
    const float* src =
        u + comp * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0] + b[0];
    float* dst = smem + comp * kp.plane + z * kp.pxy + y * kp.px;
    for (int xx = lane; xx < ext[0]; xx += 32) dst[xx] = __ldg(src + xx);
  }
}

// Sum over the 32 lanes of 32 independent values; lane l returns the total
// of v[l].  Recursive halving: 16 + 8 + 4 + 2 + 1 shuffles.
__device__ __forceinline__ float transpose_reduce32(float v[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      float send = upper ? v[i] : v[i + s];
      float keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

__global__ void __launch_bounds__(kThreads) k_gather_f32(
    erpp_kparams kp, const float* __restrict__ u, const int32_t* __restrict__ start,
    const uint32_t* __restrict__ entries, int64_t ecap, const float4* __restrict__ geo_t,
    const int4* __restrict__ geo_c, float* __restrict__ up_acc, int64_t acc_stride) {
  extern __shared__ float smem[];
  __shared__ PieceSmem ps;
  const int tile = blockIdx.x;
  const int e0 = start[tile];
  const int e1 = (int)min((int64_t)start[tile + 1], ecap);
  if (e0 >= e1) return;
  int b[3], ext[3];
  tile_origin(kp, tile, b, ext);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  stage_tile(kp, u, smem, b, ext);
  const int xs = kp.xs, R = kp.rows;
  const int ix = lane % xs, q = lane / xs;
  const bool lane_on = q < R;
  const int plane = kp.plane;
  for (int bs = e0; bs < e1; bs += kBatch) {
    const int nb = min(kBatch, e1 - bs);
    __syncthreads();  // staging done / previous batch consumed
    if ((int)threadIdx.x < nb)
      decode_piece(kp, __ldg(&entries[bs + threadIdx.x]), geo_t, geo_c, b, ext, ps,
                   threadIdx.x);
    __syncthreads();
    for (int g0 = warp * kGroup; g0 < nb; g0 += kWarps * kGroup) {
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
#pragma unroll
      for (int k = 0; k < kGroup; ++k) {
        const int j = g0 + k;
        if (j < nb && lane_on) {
          const int len = ps.len[j];
          const int lx = len & 255, ly = (len >> 8) & 255, lz = len >> 16;
          const float d0x = ps.d[0][j], d0y = ps.d[1][j], d0z = ps.d[2][j];
          const int nr = ly * lz;
          for (int xc = 0; xc < lx; xc += xs) {
            const int kx = xc + ix;
            if (kx >= lx) break;
            const float dxk = d0x + (float)kx;
            const float ex = exp2f(-kp.beta[0] * dxk * dxk);
            const float* s0 = smem + ps.base[j] + kx;
            int ky = q % ly, kz = q / ly;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
            for (int r = q; r < nr; r += R) {
              const float dy = d0y + (float)ky, dz = d0z + (float)kz;
              const float w = exp2f(-(kp.beta[1] * dy * dy + kp.beta[2] * dz * dz));
              const float* s = s0 + kz * kp.pxy + ky * kp.px;
              a0 = fmaf(w, s[0], a0);
              a1 = fmaf(w, s[plane], a1);
              a2 = fmaf(w, s[2 * plane], a2);
              ky += R;
              while (ky >= ly) {
                ky -= ly;
                ++kz;
              }
            }
            v[4 * k + 0] = fmaf(ex, a0, v[4 * k + 0]);
            v[4 * k + 1] = fmaf(ex, a1, v[4 * k + 1]);
            v[4 * k + 2] = fmaf(ex, a2, v[4 * k + 2]);
          }
        }
      }
      const float tot = transpose_reduce32(v, lane);
      const int k = lane >> 2, c = lane & 3;
      if (c < 3 && g0 + k < nb) atomicAdd(up_acc + c * acc_stride + ps.p[g0 + k], tot);
    }
  }
}

template <bool KAHAN>
__global__ void __launch_bounds__(kThreads) k_scatter_f32(
    erpp_kparams kp, float* __restrict__ S, const int32_t* __restrict__ start,
    const uint32_t* __restrict__ entries, int64_t ecap, const float4* __restrict__ geo_t,
    const int4* __restrict__ geo_c, const float4* __restrict__ fscat) {
  extern __shared__ float smem[];
  __shared__ PieceSmem ps;
  __shared__ float red[kWarps];
  const int tile = blockIdx.x;
  const int e0 = start[tile];
  const int e1 = (int)min((int64_t)start[tile + 1], ecap);
  int b[3], ext[3];
  tile_origin(kp, tile, b, ext);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int plane = kp.plane;
  const bool any = e0 < e1;
  // Tiles with many pieces (dense clusters) accumulate in compensated FP32:
  // there the fixed-point bound sum(max|f|) is far above the node values
  // whenever signs cancel.  Needs the 6-plane allocation of the Kahan mode.
  const bool comp = KAHAN || (kp.kahan_alloc && (e1 - e0) > kDenseTile);
  float scale = 1.f, inv_scale = 1.f;
  if (any) {
    const int total = (comp ? 6 : 3) * plane;
    for (int k = threadIdx.x; k < total; k += kThreads) smem[k] = 0.f;
    if (!comp) {
      // B = sum over the tile's pieces of max_c |f_c| (kept in fscat.w)
      float bsum = 0.f;
      for (int e = e0 + threadIdx.x; e < e1; e += kThreads)
        bsum += __ldg(&fscat[__ldg(&entries[e]) & ERPP_ENTRY_PMASK]).w;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
      if (lane == 0) red[warp] = bsum;
      __syncthreads();
      float B = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) B += red[w];
      if (B > 0.f) {
        int ex;
        frexpf(B, &ex);  // B = m 2^ex, m in [0.5, 1)
        int sh = min(30 - ex, 120);
        scale = ldexpf(1.f, sh);
        inv_scale = ldexpf(1.f, -sh);
      }
    }
    const int xs = kp.xs, R = kp.rows;
    const int ix = lane % xs, q = lane / xs;
    const bool lane_on = q < R;
    int* acc_i = reinterpret_cast<int*>(smem);
    float* comp_lo = smem + 3 * plane;
    for (int bs = e0; bs < e1; bs += kBatch) {
      const int nb = min(kBatch, e1 - bs);
      __syncthreads();
      if ((int)threadIdx.x < nb) {
        const uint32_t word = __ldg(&entries[bs + threadIdx.x]);
        decode_piece(kp, word, geo_t, geo_c, b, ext, ps, threadIdx.x);
        const float4 f = __ldg(&fscat[word & ERPP_ENTRY_PMASK]);
        ps.f[0][threadIdx.x] = f.x * scale;
        ps.f[1][threadIdx.x] = f.y * scale;
        ps.f[2][threadIdx.x] = f.z * scale;
      }
      __syncthreads();
      if (!lane_on) continue;
      for (int j = warp; j < nb; j += kWarps) {
        const int len = ps.len[j];
        const int lx = len & 255, ly = (len >> 8) & 255, lz = len >> 16;
        const float d0x = ps.d[0][j], d0y = ps.d[1][j], d0z = ps.d[2][j];
        const float f0 = ps.f[0][j], f1 = ps.f[1][j], f2 = ps.f[2][j];
        const int nr = ly * lz;
        for (int xc = 0; xc < lx; xc += xs) {
          const int kx = xc + ix;
          if (kx >= lx) break;
          const float dxk = d0x + (float)kx;
          const float ex = exp2f(-kp.beta[0] * dxk * dxk);
          const float g0 = f0 * ex, g1 = f1 * ex, g2 = f2 * ex;
          const int i0 = ps.base[j] + kx;
          int ky = q % ly, kz = q / ly;
          for (int r = q; r < nr; r += R) {
            const float dy = d0y + (float)ky, dz = d0z + (float)kz;
            const float w = exp2f(-(kp.beta[1] * dy * dy + kp.beta[2] * dz * dz));
            const int idx = i0 + kz * kp.pxy + ky * kp.px;
            if (comp) {
              const float vals[3] = {g0 * w, g1 * w, g2 * w};
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const float vv = vals[c];
                const float old = atomicAdd(smem + c * plane + idx, vv);
                const float s = old + vv;
                const float bp = s - old;
                const float err = (old - (s - bp)) + (vv - bp);
                atomicAdd(comp_lo + c * plane + idx, err);
              }
            } else {
              atomicAdd(acc_i + idx, __float2int_rn(g0 * w));
              atomicAdd(acc_i + plane + idx, __float2int_rn(g1 * w));
              atomicAdd(acc_i + 2 * plane + idx, __float2int_rn(g2 * w));
            }
            ky += R;
            while (ky >= ly) {
              ky -= ly;
              ++kz;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // write the interior once (zeros for empty tiles)
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int nrow = 3 * ext[1] * ext[2];
  const int* acc_i = reinterpret_cast<const int*>(smem);
  for (int r = warp; r < nrow; r += kWarps) {
    int cc = r / (ext[1] * ext[2]);
    int yz = r - cc * ext[1] * ext[2];
    int z = yz / ext[1];
    int y = yz - z * ext[1];
    float* dst = S + cc * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0] + b[0];
    const int so = cc * plane + z * kp.pxy + y * kp.px;
    for (int xx = lane; xx < ext[0]; xx += 32) {
      float val = 0.f;
      if (any) {
        if (comp)
          val = smem[so + xx] + smem[3 * plane + so + xx];
        else
          val = (float)acc_i[so + xx] * inv_scale;
      }
      dst[xx] = val;
    }
  }
}

size_t tile_smem_bytes(const erpp_kparams& kp, bool two) {
  return sizeof(float) * (size_t)kp.plane * (two ? 6 : 3);
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
  k_gather_f32<<<kp.ntiles, kThreads, sm, st>>>(kp, u, ctx->tile_start, ctx->entries,
                                                ctx->entries_cap, ctx->geo_t, ctx->geo_c,
                                                ctx->up_acc, ctx->cap);
  return cudaGetLastError();
}

cudaError_t launch_scatter_f32(erpp_ctx* ctx, float* S, cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  const bool kahan = kp.kahan != 0;
  size_t sm = tile_smem_bytes(kp, kahan || kp.kahan_alloc);
  cudaError_t e;
  if (kahan) {
    e = cudaFuncSetAttribute(k_scatter_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    k_scatter_f32<true><<<kp.ntiles, kThreads, sm, st>>>(kp, S, ctx->tile_start, ctx->entries,
                                                         ctx->entries_cap, ctx->geo_t,
                                                         ctx->geo_c, ctx->fscat);
  } else {
    e = cudaFuncSetAttribute(k_scatter_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    k_scatter_f32<false><<<kp.ntiles, kThreads, sm, st>>>(kp, S, ctx->tile_start, ctx->entries,
                                                          ctx->entries_cap, ctx->geo_t,
                                                          ctx->geo_c, ctx->fscat);
  }
  return cudaGetLastError();
}

}  // namespace erpp
