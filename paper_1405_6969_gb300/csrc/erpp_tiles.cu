// erpp_tiles.cu -- FP32 tile kernels: the kernel gather and the regularised
// source scatter (Sec. 2.4, Eq. ns_regularized_filtered; the heat kernel of
// App. A.1 factored per axis).
//
// One thread block owns one grid tile and stages it in shared memory as
// [3][T_z][T_y][96]: a row holds the tile's x-range (64 nodes) plus an x-halo
// of hlo nodes below and hhi above, so that every particle whose home cell
// lies in the tile finds its whole x-window in the row.  Rows are 96 floats,
// a multiple of the 32 banks, so the bank of a node is its local x' mod 32
// whatever its row.
//
// The binning sorts a tile's pieces (a particle's window cut to the tile's
// y/z range) into 32 buckets by x0 mod 32, x0 the first local x' of the piece,
// and precomputes each piece's record (first node, window lengths, distances)
// and each particle's x-weights.  Lane l of every warp takes pieces from
// bucket l (a shared-memory queue per bucket, so the eight warps share a
// bucket's work dynamically) and, once that bucket is empty, from the next
// non-empty one.  A lane owns its piece: it walks the piece's rows (y, z) one
// per iteration and reads or updates the row's nodes x0 .. x0 + lx - 1 in
// order, so at each step the 32 lanes touch 32 different banks (while they
// work on their own buckets) and the gather needs no reduction across lanes.
// The next piece's record is loaded while the current one is processed.
// Weights are separable:
//   w = 2^(-beta_x d_x^2) * 2^(-(beta_y d_y^2 + beta_z d_z^2)),
// d in grid units from the particle, beta = log2(e) dx^2 / (2 sigma_R^2): the
// x factors come with the particle, one exponential per row.
//
// Gather: a lane sums w*u over its piece and adds the three totals to the
// particle's accumulator in global memory; normalisation is applied later.
//
// Scatter: contributions are accumulated exactly in 32-bit fixed point with
// shared-memory integer atomics (order independent, hence deterministic).
// The tile's scale is the power of two 2^30 / B, B >= the sum over its pieces
// of max|f|, which bounds every node (unnormalised weights are <= 1), so no sum
// overflows.  A piece's force times its x-weights is rounded to integers G
// once per piece, the row weight to W = round(w 2^24) once per row, and each
// node receives round(G W 2^-24) (one integer multiply, no float-to-integer
// conversion per node); the error per contribution is about B 2^-30.  Tiles
// with more than 1024 pieces (dense clusters, where signs cancel far below B)
// add FP32 values with shared atomics instead.  With ERPP_KAHAN every tile
// adds FP32 values and keeps the exact rounding error of each addition
// (two-sum on the value the atomic returned) in a second array.  The tile's
// interior is written to HBM once, zeros included; its halo columns go to a
// small buffer that k_merge_halo adds onto the neighbouring tiles afterwards.
#include <cuda_runtime.h>

#include <algorithm>

#include "erpp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kDenseTile = 1024;  // pieces above which a tile accumulates in FP32

struct Piece {
  int p;            // particle
  int lx, ly, lz;   // window lengths (x whole, y/z clipped to the tile)
  int base;         // shared-memory index of the first node
  float d0y, d0z;   // distances (grid units) of the first y and z nodes
};

__device__ __forceinline__ void tile_origin(const erpp_kparams& kp, int tile, int b[3],
                                            int ext[3]) {
  const int txy = kp.nt[0] * kp.nt[1];
  const int tz = tile / txy;
  const int r = tile - tz * txy;
  const int ty = r / kp.nt[0];
  const int tx = r - ty * kp.nt[0];
  b[0] = tx * kp.T[0];
  b[1] = ty * kp.T[1];
  b[2] = tz * kp.T[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) ext[a] = min(b[a] + kp.T[a], kp.n[a]) - b[a];
}

__device__ __forceinline__ void unpack_piece(int4 rec, Piece& pc) {
  pc.p = rec.x;
  const uint32_t v = (uint32_t)rec.y;
  pc.base = (int)(v & ((1u << ERPP_BASE_BITS) - 1u));
  pc.lx = (int)((v >> 17) & 31u);
  pc.ly = (int)((v >> 22) & 31u);
  pc.lz = (int)(v >> 27);
  pc.d0y = __int_as_float(rec.z);
  pc.d0z = __int_as_float(rec.w);
}

template <int XW>
__device__ __forceinline__ void load_xw(const float* __restrict__ xw, int p,
                                        float4 (&o)[XW / 4]) {
  const float4* src = reinterpret_cast<const float4*>(xw + (size_t)p * XW);
#pragma unroll
  for (int k = 0; k < XW / 4; ++k) o[k] = __ldg(src + k);
}

// Per-bucket work queues of one tile: lane l pops from bucket l, then from
// the following buckets once l is exhausted.  Returns an entry index or -1.
struct Queues {
  int next[32];
  int end[32];
};

__device__ __forceinline__ int pop_entry(Queues& qs, int& bkt) {
  for (int tries = 0; tries < 32; ++tries) {
    const int e = atomicAdd(&qs.next[bkt], 1);
    if (e < qs.end[bkt]) return e;
    bkt = (bkt + 1) & 31;
  }
  return -1;
}

__device__ __forceinline__ void init_queues(Queues& qs, const int32_t* __restrict__ start,
                                            int tile, int64_t ecap) {
  const int tid = threadIdx.x;
  if (tid < 32) {
    qs.next[tid] = start[tile * 32 + tid];
    qs.end[tid] = (int)min((int64_t)start[tile * 32 + tid + 1], ecap);
  }
}

__device__ __forceinline__ void stage_tile(const erpp_kparams& kp, const float* __restrict__ u,
                                           float* smem, const int b[3], const int ext[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int nrow = 3 * ext[1] * ext[2];
  const int width = ext[0] + kp.xhlo + kp.xhhi;
  const int gx0 = b[0] - kp.xhlo;
  for (int r = warp; r < nrow; r += kWarps) {
    const int comp = r / (ext[1] * ext[2]);
    const int yz = r - comp * ext[1] * ext[2];
    const int z = yz / ext[1];
    const int y = yz - z * ext[1];
    const float* src = u + comp * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0];
    float* dst = smem + comp * kp.plane + z * kp.pxy + y * kp.px;
    for (int xx = lane; xx < kp.px; xx += 32) {
      float v = 0.f;
      if (xx < width) {
        int gx = gx0 + xx;
        gx = gx < 0 ? gx + kp.n[0] : (gx >= kp.n[0] ? gx - kp.n[0] : gx);
        v = __ldg(src + gx);
      }
      dst[xx] = v;
    }
  }
}

// XM: longest x-window; LMIN: shortest (the x-window is never cut, so only
// the slots q >= LMIN need a test); XW: x-weights stored per particle.
template <int XM, int LMIN, int XW>
__global__ void __launch_bounds__(kThreads) k_gather_f32(
    erpp_kparams kp, const float* __restrict__ u, const int32_t* __restrict__ start,
    const int4* __restrict__ entries, int64_t ecap, const float* __restrict__ xw,
    float* __restrict__ up_acc, int64_t acc_stride) {
  extern __shared__ float smem[];
  __shared__ Queues qs;
  const int tile = blockIdx.x;
  if (start[tile * 32] >= (int)min((int64_t)start[tile * 32 + 32], ecap)) return;
  int b[3], ext[3];
  tile_origin(kp, tile, b, ext);
  stage_tile(kp, u, smem, b, ext);
  init_queues(qs, start, tile, ecap);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int plane = kp.plane, px = kp.px, pxy = kp.pxy;
  const float by = kp.beta[1], bz = kp.beta[2];
  int bkt = lane;
  // record and x-weights of the next piece, loaded while the current one runs
  int4 rn = make_int4(0, 0, 0, 0);
  float4 xn[XW / 4];
  int en = pop_entry(qs, bkt);
  if (en >= 0) {
    rn = __ldg(&entries[en]);
    load_xw<XW>(xw, rn.x, xn);
  }
  Piece pc;
  float ex[XW];
  int iy = 0, iz = 0;
  float dyf = 0.f, ezz = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
  const float* srow = smem;
  bool have = false;
  auto next_piece = [&]() {
    have = en >= 0;
    if (!have) return;
    unpack_piece(rn, pc);
#pragma unroll
    for (int k = 0; k < XW / 4; ++k) {
      ex[4 * k] = xn[k].x;
      ex[4 * k + 1] = xn[k].y;
      ex[4 * k + 2] = xn[k].z;
      ex[4 * k + 3] = xn[k].w;
    }
    iy = 0;
    iz = 0;
    dyf = pc.d0y;
    ezz = bz * pc.d0z * pc.d0z;
    srow = smem + pc.base;
    a0 = a1 = a2 = 0.f;
    en = pop_entry(qs, bkt);
    if (en >= 0) {
      rn = __ldg(&entries[en]);
      load_xw<XW>(xw, rn.x, xn);
    }
  };
  next_piece();
  while (__any_sync(0xffffffffu, have)) {
    if (have) {
      const float w = exp2f(-fmaf(by * dyf, dyf, ezz));
      float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
      for (int q = 0; q < XM; ++q) {
        if (q < LMIN || q < pc.lx) {
          r0 = fmaf(ex[q], srow[q], r0);
          r1 = fmaf(ex[q], srow[q + plane], r1);
          r2 = fmaf(ex[q], srow[q + 2 * plane], r2);
        }
      }
      a0 = fmaf(w, r0, a0);
      a1 = fmaf(w, r1, a1);
      a2 = fmaf(w, r2, a2);
      srow += px;
      dyf += 1.f;
      if (++iy == pc.ly) {
        iy = 0;
        dyf = pc.d0y;
        srow += pxy - pc.ly * px;
        const float dz = pc.d0z + (float)(++iz);
        ezz = bz * dz * dz;
        if (iz == pc.lz) {
          atomicAdd(up_acc + pc.p, a0);
          atomicAdd(up_acc + acc_stride + pc.p, a1);
          atomicAdd(up_acc + 2 * acc_stride + pc.p, a2);
          next_piece();
        }
      }
    }
  }
}

// MODE 0: fixed point (FP32 atomics on dense tiles); MODE 1: compensated FP32.
template <int XM, int LMIN, int XW, int MODE>
__global__ void __launch_bounds__(kThreads) k_scatter_f32(
    erpp_kparams kp, float* __restrict__ S, float* __restrict__ halo,
    const int32_t* __restrict__ start, const int4* __restrict__ entries, int64_t ecap,
    const float* __restrict__ xw, const float4* __restrict__ fscat) {
  extern __shared__ float smem[];
  __shared__ Queues qs;
  __shared__ float red[kWarps];
  const int tile = blockIdx.x;
  const int e0 = start[tile * 32];
  const int e1 = (int)min((int64_t)start[tile * 32 + 32], ecap);
  int b[3], ext[3];
  tile_origin(kp, tile, b, ext);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int plane = kp.plane, px = kp.px, pxy = kp.pxy;
  const bool any = e0 < e1;
  const bool fixedp = MODE == 0 && (e1 - e0) <= kDenseTile;
  float scale = 1.f, inv_scale = 1.f;
  if (any) {
    const int total = (MODE == 1 ? 6 : 3) * plane;
    for (int k = threadIdx.x; k < total; k += kThreads) smem[k] = 0.f;
    init_queues(qs, start, tile, ecap);
    if (fixedp) {
      // B = sum over the tile's pieces of max_c |f_c| (kept in fscat.w)
      float bsum = 0.f;
      for (int e = e0 + threadIdx.x; e < e1; e += kThreads)
        bsum += __ldg(&fscat[__ldg(&entries[e].x)]).w;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
      if (lane == 0) red[warp] = bsum;
    }
    __syncthreads();
    if (fixedp) {
      float B = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) B += red[w];
      if (B > 0.f) {
        int ex;
        frexpf(B, &ex);  // B = m 2^ex, m in [0.5, 1)
        const int sh = min(30 - ex, 120);
        scale = ldexpf(1.f, sh);
        inv_scale = ldexpf(1.f, -sh);
      }
    }
    int* acc_i = reinterpret_cast<int*>(smem);
    float* comp_lo = smem + 3 * plane;
    const float by = kp.beta[1], bz = kp.beta[2];
    int bkt = lane;
    int4 rn = make_int4(0, 0, 0, 0);
    float4 xn[XW / 4];
    float4 fn = make_float4(0.f, 0.f, 0.f, 0.f);
    int en = pop_entry(qs, bkt);
    if (en >= 0) {
      rn = __ldg(&entries[en]);
      load_xw<XW>(xw, rn.x, xn);
      fn = __ldg(&fscat[rn.x]);
    }
    Piece pc;
    float ex[XM];                  // x-weights
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    int G0[XM], G1[XM], G2[XM];    // force times x-weight, fixed point
    int iy = 0, iz = 0, row = 0;
    float dyf = 0.f, ezz = 0.f;
    bool have = false;
    auto next_piece = [&]() {
      have = en >= 0;
      if (!have) return;
      unpack_piece(rn, pc);
      float exw[XW];
#pragma unroll
      for (int k = 0; k < XW / 4; ++k) {
        exw[4 * k] = xn[k].x;
        exw[4 * k + 1] = xn[k].y;
        exw[4 * k + 2] = xn[k].z;
        exw[4 * k + 3] = xn[k].w;
      }
      f0 = fn.x * scale;
      f1 = fn.y * scale;
      f2 = fn.z * scale;
#pragma unroll
      for (int q = 0; q < XM; ++q) {
        ex[q] = exw[q];
        if (MODE == 0 && fixedp) {
          G0[q] = __float2int_rn(f0 * exw[q]);
          G1[q] = __float2int_rn(f1 * exw[q]);
          G2[q] = __float2int_rn(f2 * exw[q]);
        }
      }
      iy = 0;
      iz = 0;
      dyf = pc.d0y;
      ezz = bz * pc.d0z * pc.d0z;
      row = pc.base;
      en = pop_entry(qs, bkt);
      if (en >= 0) {
        rn = __ldg(&entries[en]);
        load_xw<XW>(xw, rn.x, xn);
        fn = __ldg(&fscat[rn.x]);
      }
    };
    next_piece();
    while (__any_sync(0xffffffffu, have)) {
      if (have) {
        const float w = exp2f(-fmaf(by * dyf, dyf, ezz));
        if (MODE == 1) {
#pragma unroll
          for (int q = 0; q < XM; ++q) {
            if (q < LMIN || q < pc.lx) {
              const float wq = w * ex[q];
              const float vals[3] = {f0 * wq, f1 * wq, f2 * wq};
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const float vv = vals[c];
                const float old = atomicAdd(smem + c * plane + row + q, vv);
                const float s = old + vv;
                const float bp = s - old;
                const float err = (old - (s - bp)) + (vv - bp);
                atomicAdd(comp_lo + c * plane + row + q, err);
              }
            }
          }
        } else if (fixedp) {
          const long long W = (long long)__float2int_rn(w * 16777216.f);
#pragma unroll
          for (int q = 0; q < XM; ++q) {
            if (q < LMIN || q < pc.lx) {
              atomicAdd(acc_i + row + q, (int)(((long long)G0[q] * W + 8388608LL) >> 24));
              atomicAdd(acc_i + plane + row + q,
                        (int)(((long long)G1[q] * W + 8388608LL) >> 24));
              atomicAdd(acc_i + 2 * plane + row + q,
                        (int)(((long long)G2[q] * W + 8388608LL) >> 24));
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < XM; ++q) {
            if (q < LMIN || q < pc.lx) {
              const float wq = w * ex[q];
              atomicAdd(smem + row + q, f0 * wq);
              atomicAdd(smem + plane + row + q, f1 * wq);
              atomicAdd(smem + 2 * plane + row + q, f2 * wq);
            }
          }
        }
        row += px;
        dyf += 1.f;
        if (++iy == pc.ly) {
          iy = 0;
          dyf = pc.d0y;
          row += pxy - pc.ly * px;
          const float dz = pc.d0z + (float)(++iz);
          ezz = bz * dz * dz;
          if (iz == pc.lz) next_piece();
        }
      }
    }
    __syncthreads();
  }
  // write the interior once (zeros for empty tiles), and the halo columns
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int hw = kp.xhlo + kp.xhhi;
  const int nrow = 3 * ext[1] * ext[2];
  const int* acc_i = reinterpret_cast<const int*>(smem);
  for (int r = warp; r < nrow; r += kWarps) {
    const int cc = r / (ext[1] * ext[2]);
    const int yz = r - cc * ext[1] * ext[2];
    const int z = yz / ext[1];
    const int y = yz - z * ext[1];
    float* dst = S + cc * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0] + b[0];
    float* hdst = halo + ((((size_t)tile * 3 + cc) * kp.T[2] + z) * kp.T[1] + y) * hw;
    const int so = cc * plane + z * pxy + y * px;
    const int width = ext[0] + hw;
    for (int xx = lane; xx < width; xx += 32) {
      float val = 0.f;
      if (any) {
        if (MODE == 1)
          val = smem[so + xx] + smem[3 * plane + so + xx];
        else if (fixedp)
          val = (float)acc_i[so + xx] * inv_scale;
        else
          val = smem[so + xx];
      }
      if (xx < kp.xhlo)
        hdst[xx] = val;
      else if (xx < kp.xhlo + ext[0])
        dst[xx - kp.xhlo] = val;
      else
        hdst[xx - ext[0]] = val;
    }
  }
}

// Adds the scatter's x-halo columns onto the tiles they belong to: column i of
// tile t receives the right halo of tile t-1 (i < hhi) and the left halo of
// tile t+1 (i >= width - hlo), periodic in x.  One thread per node, one write.
// Needs every tile at least max(hlo, hhi) wide (checked at initialisation).
__global__ void k_merge_halo(erpp_kparams kp, float* __restrict__ S,
                             const float* __restrict__ halo) {
  const int hw = kp.xhlo + kp.xhhi;
  const int64_t per_tile = 3LL * kp.T[2] * kp.T[1] * hw;
  const int64_t total = per_tile * kp.ntiles;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int tile = (int)(g / per_tile);
    int64_t r = g - (int64_t)tile * per_tile;
    const int col = (int)(r % hw);
    r /= hw;
    const int y = (int)(r % kp.T[1]);
    r /= kp.T[1];
    const int z = (int)(r % kp.T[2]);
    const int cc = (int)(r / kp.T[2]);
    int b[3], ext[3];
    tile_origin(kp, tile, b, ext);
    if (y >= ext[1] || z >= ext[2]) continue;
    const int W = ext[0];
    if (col >= min(W, hw)) continue;
    const int i = (W >= hw && col >= kp.xhhi) ? W - kp.xhlo + (col - kp.xhhi) : col;
    const int txy = kp.nt[0] * kp.nt[1];
    const int tz = tile / txy;
    const int ty = (tile - tz * txy) / kp.nt[0];
    const int tx = tile - tz * txy - ty * kp.nt[0];
    const int trow = kp.nt[0] * (ty + kp.nt[1] * tz);
    const int tl = (tx == 0 ? kp.nt[0] - 1 : tx - 1) + trow;
    const int tr = (tx == kp.nt[0] - 1 ? 0 : tx + 1) + trow;
    float add = 0.f;
    if (i < kp.xhhi)
      add += halo[((((size_t)tl * 3 + cc) * kp.T[2] + z) * kp.T[1] + y) * hw + kp.xhlo + i];
    if (i >= W - kp.xhlo)
      add += halo[((((size_t)tr * 3 + cc) * kp.T[2] + z) * kp.T[1] + y) * hw +
                  (i - (W - kp.xhlo))];
    float* dst = S + cc * nn + ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y)) * kp.n[0] + b[0] + i;
    *dst += add;
  }
}

size_t tile_smem_bytes(const erpp_kparams& kp, bool two) {
  return sizeof(float) * (size_t)kp.plane * (two ? 6 : 3);
}

template <int XM, int LMIN, int XW>
cudaError_t gather_xm(erpp_ctx* ctx, const float* u, cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  const size_t sm = tile_smem_bytes(kp, false);
  cudaError_t e = cudaFuncSetAttribute(k_gather_f32<XM, LMIN, XW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ++ctx->launches;
  k_gather_f32<XM, LMIN, XW><<<kp.ntiles, kThreads, sm, st>>>(
      kp, u, ctx->tile_start, ctx->entries, ctx->entries_cap, ctx->xw, ctx->up_acc, ctx->cap);
  return cudaGetLastError();
}

template <int XM, int LMIN, int XW, int MODE>
cudaError_t scatter_xm(erpp_ctx* ctx, float* S, cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  const size_t sm = tile_smem_bytes(kp, MODE == 1);
  cudaError_t e = cudaFuncSetAttribute(k_scatter_f32<XM, LMIN, XW, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ++ctx->launches;
  k_scatter_f32<XM, LMIN, XW, MODE><<<kp.ntiles, kThreads, sm, st>>>(
      kp, S, ctx->halo, ctx->tile_start, ctx->entries, ctx->entries_cap, ctx->xw, ctx->fscat);
  return cudaGetLastError();
}

template <int XM, int LMIN, int XW>
cudaError_t scatter_k(erpp_ctx* ctx, float* S, cudaStream_t st) {
  return ctx->kp.kahan ? scatter_xm<XM, LMIN, XW, 1>(ctx, S, st)
                       : scatter_xm<XM, LMIN, XW, 0>(ctx, S, st);
}

// Specialised window lengths: x-windows of 6-7 nodes (cutoff 3 sigma_R at
// sigma_R = dx; 5-7 when rounding leaves c' just below 3) and 9-10 nodes
// (sigma_R = 1.5 dx); other windows of up to 16 nodes take a generic variant
// that tests every slot.  The x-weight record length follows the variant.
int variant(const erpp_kparams& kp) {
  if (kp.xxs <= 7 && kp.xlmin >= 6) return 0;
  if (kp.xxs <= 7 && kp.xlmin >= 5) return 1;
  if (kp.xxs <= 10 && kp.xlmin >= 9) return 2;
  if (kp.xxs <= 10 && kp.xlmin >= 8) return 3;
  return 4;
}

}  // namespace

namespace erpp {

// Length of the per-particle x-weight record for a parameter set.
int xw_len(const erpp_kparams& kp) { return variant(kp) <= 1 ? 8 : 16; }

cudaError_t launch_gather_f32(erpp_ctx* ctx, const float* u, int64_t n, cudaStream_t st) {
  (void)n;
  if (ctx->kp.design == 4) return launch_gather_f32_4(ctx, u, st);
  switch (variant(ctx->kp)) {
    case 0: return gather_xm<7, 6, 8>(ctx, u, st);
    case 1: return gather_xm<7, 5, 8>(ctx, u, st);
    case 2: return gather_xm<10, 9, 16>(ctx, u, st);
    case 3: return gather_xm<10, 8, 16>(ctx, u, st);
    default: return gather_xm<16, 1, 16>(ctx, u, st);
  }
}

cudaError_t launch_scatter_f32(erpp_ctx* ctx, float* S, cudaStream_t st) {
  if (ctx->kp.design == 4) return launch_scatter_f32_4(ctx, S, st);
  cudaError_t e;
  switch (variant(ctx->kp)) {
    case 0: e = scatter_k<7, 6, 8>(ctx, S, st); break;
    case 1: e = scatter_k<7, 5, 8>(ctx, S, st); break;
    case 2: e = scatter_k<10, 9, 16>(ctx, S, st); break;
    case 3: e = scatter_k<10, 8, 16>(ctx, S, st); break;
    default: e = scatter_k<16, 1, 16>(ctx, S, st); break;
  }
  if (e != cudaSuccess) return e;
  const erpp_kparams& kp = ctx->kp;
  const int64_t total = 3LL * kp.T[2] * kp.T[1] * (kp.xhlo + kp.xhhi) * kp.ntiles;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  ++ctx->launches;
  k_merge_halo<<<blocks, 256, 0, st>>>(kp, S, ctx->halo);
  return cudaGetLastError();
}

}  // namespace erpp
