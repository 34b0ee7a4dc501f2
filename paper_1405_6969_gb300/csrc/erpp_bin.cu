// erpp_bin.cu -- binning of particles into grid tiles (device counting sort).
//
// Each particle's truncated stencil (a box of at most xs^3 nodes, Sec. 2.4:
// the forcing of a particle reaches only the nodes within a few sigma_R) is
// split along tile boundaries and periodic images into (tile, shift) pieces.
// One "entry" per piece is written, grouped by tile, so that the gather and
// the scatter can both work on one tile interior per thread block with no
// halo and no wrap-around in shared memory.
//
// Passes: k_bin_count (geometry per particle + per-tile piece counts),
// k_scan (exclusive scan of the counts), k_bin_fill (place the entries).
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

// Calls f(tile, code) for every (tile, periodic shift) piece of the window
// [jlo, jlo + nw - 1] per axis (unwrapped node indices).
template <typename F>
__device__ __forceinline__ void for_each_piece(const erpp_kparams& kp, const int jlo[3],
                                               const int nw[3], F f) {
  const int jhx = jlo[0] + nw[0] - 1, jhy = jlo[1] + nw[1] - 1, jhz = jlo[2] + nw[2] - 1;
  for (int jx = jlo[0]; jx <= jhx;) {
    int mx = erpp_floordiv(jx, kp.n[0]);
    int wx = jx - mx * kp.n[0];
    int tx = wx / kp.T[0];
    int ex = min(min((tx + 1) * kp.T[0], kp.n[0]) - wx + jx - 1, jhx);
    for (int jy = jlo[1]; jy <= jhy;) {
      int my = erpp_floordiv(jy, kp.n[1]);
      int wy = jy - my * kp.n[1];
      int ty = wy / kp.T[1];
      int ey = min(min((ty + 1) * kp.T[1], kp.n[1]) - wy + jy - 1, jhy);
      for (int jz = jlo[2]; jz <= jhz;) {
        int mz = erpp_floordiv(jz, kp.n[2]);
        int wz = jz - mz * kp.n[2];
        int tz = wz / kp.T[2];
        int ez = min(min((tz + 1) * kp.T[2], kp.n[2]) - wz + jz - 1, jhz);
        int tile = (tz * kp.nt[1] + ty) * kp.nt[0] + tx;
        uint32_t code = (uint32_t)((mx + 1) + 3 * (my + 1) + 9 * (mz + 1));
        f(tile, code);
        jz = ez + 1;
      }
      jy = ey + 1;
    }
    jx = ex + 1;
  }
}

__global__ void k_bin_count(erpp_kparams kp, int64_t n, const double* __restrict__ x0,
                            const double* __restrict__ x1, const double* __restrict__ x2,
                            float4* __restrict__ geo_t, int4* __restrict__ geo_c,
                            float* __restrict__ up_acc, int64_t acc_stride,
                            int32_t* __restrict__ tile_cnt, uint32_t* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xv[3] = {x0[i], x1[i], x2[i]};
  if (up_acc) {
    up_acc[i] = 0.f;
    up_acc[acc_stride + i] = 0.f;
    up_acc[2 * acc_stride + i] = 0.f;
  }
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) ok = ok && (xv[a] >= 0.0) && (xv[a] < kp.L[a]);
  if (!ok) {
    erpp_set_err(err, ERPP_ERRBIT_RANGE);
    geo_t[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    geo_c[i] = make_int4(0, 0, 0, 0);
    return;
  }
  int c[3], off[3], nw[3], jlo[3];
  float t[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double s, lo, hi;
    erpp_axis_window(xv[a], kp.inv_dx[a], kp.cp[a], &s, &lo, &hi);
    double fl = floor(s);
    int ci = (int)fl;
    off[a] = (int)lo - ci;
    nw[a] = (int)hi - (int)lo + 1;
    t[a] = (float)__dadd_rn(s, -fl);
    // s can round up to exactly N for x just below L: the cell is then the
    // first one of the next image, which is the same node set shifted by N.
    if (ci >= kp.n[a]) ci -= kp.n[a];
    c[a] = ci;
    jlo[a] = ci + off[a];
    ok = ok && off[a] >= -kp.hlo && off[a] <= 0 && nw[a] >= 1 && nw[a] <= kp.xs;
  }
  if (!ok) {
    erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
    geo_t[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    geo_c[i] = make_int4(0, 0, 0, 0);
    return;
  }
  uint32_t pack = ERPP_GEO_VALID;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    pack |= (uint32_t)(-off[a]) << (4 * a);
    pack |= (uint32_t)nw[a] << (12 + 5 * a);
  }
  geo_t[i] = make_float4(t[0], t[1], t[2], 0.f);
  geo_c[i] = make_int4(c[0], c[1], c[2], (int)pack);
  for_each_piece(kp, jlo, nw, [&](int tile, uint32_t) { atomicAdd(&tile_cnt[tile], 1); });
}

__global__ void k_bin_fill(erpp_kparams kp, int64_t n, const int4* __restrict__ geo_c,
                           int32_t* __restrict__ cursor, uint32_t* __restrict__ entries,
                           int64_t cap, uint32_t* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int4 g = geo_c[i];
  uint32_t pack = (uint32_t)g.w;
  if (!(pack & ERPP_GEO_VALID)) return;
  int c[3] = {g.x, g.y, g.z};
  int jlo[3], nw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    jlo[a] = c[a] + erpp_geo_off(pack, a);
    nw[a] = erpp_geo_nw(pack, a);
  }
  for_each_piece(kp, jlo, nw, [&](int tile, uint32_t code) {
    int pos = atomicAdd(&cursor[tile], 1);
    if (pos < cap)
      entries[pos] = (uint32_t)i | (code << ERPP_ENTRY_PBITS);
    else
      erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
  });
}

// Exclusive scan of the per-tile counts by one thread block.
__global__ void k_scan(const int32_t* __restrict__ cnt, int32_t* __restrict__ start,
                       int32_t* __restrict__ cursor, int ntiles) {
  __shared__ int32_t warp_sums[32];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int chunk = (ntiles + nthr - 1) / nthr;
  const int lo = min(tid * chunk, ntiles), hi = min(lo + chunk, ntiles);
  int32_t local = 0;
  for (int k = lo; k < hi; ++k) local += cnt[k];
  // block-wide exclusive scan of the per-thread sums
  const int lane = tid & 31, warp = tid >> 5;
  int32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t ws = (lane < (nthr >> 5)) ? warp_sums[lane] : 0;
    int32_t wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    warp_sums[lane] = wi - ws;
  }
  __syncthreads();
  int32_t run = warp_sums[warp] + incl - local;
  for (int k = lo; k < hi; ++k) {
    start[k] = run;
    cursor[k] = run;
    run += cnt[k];
  }
  if (tid == nthr - 1) start[ntiles] = run;
}

}  // namespace

namespace erpp {

cudaError_t bin_particles(erpp_ctx* ctx, int64_t n, const double* const x[3], bool zero_acc,
                          cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  cudaError_t e = cudaMemsetAsync(ctx->tile_cnt, 0, sizeof(int32_t) * kp.ntiles, st);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    int blocks = (int)((n + 255) / 256);
    k_bin_count<<<blocks, 256, 0, st>>>(kp, n, x[0], x[1], x[2], ctx->geo_t, ctx->geo_c,
                                        zero_acc ? ctx->up_acc : nullptr, ctx->cap,
                                        ctx->tile_cnt, ctx->err);
  }
  k_scan<<<1, 1024, 0, st>>>(ctx->tile_cnt, ctx->tile_start, ctx->tile_cursor, kp.ntiles);
  if (n > 0) {
    int blocks = (int)((n + 255) / 256);
    k_bin_fill<<<blocks, 256, 0, st>>>(kp, n, ctx->geo_c, ctx->tile_cursor, ctx->entries,
                                       ctx->entries_cap, ctx->err);
  }
  return cudaGetLastError();
}

}  // namespace erpp
