// erpp_bin.cu -- binning of particles into grid tiles (device counting sort).
//
// Each particle's truncated stencil (a box of at most xs^3 nodes, Sec. 2.4:
// the forcing of a particle reaches only the nodes within a few sigma_R) is
// assigned to the x-tile of its home cell and split along y/z tile
// boundaries and periodic images into (tile, shift) pieces.  One "entry" per
// piece is written, grouped by tile, so that the gather and the scatter can
// both work on one staged tile per thread block.
//
// Passes: k_bin_count (geometry per particle; each piece takes the next
// place in its bin with one atomic increment of the bin's count and keeps
// it), k_scan (exclusive scan of the counts), k_bin_fill (each piece's record
// written at its bin's start plus its place, no atomics).
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

// One piece of a particle's stencil: the y/z window part [jy, ey] x [jz, ez]
// (unwrapped node indices) inside tile (tx, ty, tz) at periodic image
// (my, mz).
struct PieceSeg {
  int tx, ty, tz;
  int jy, ey, my, jz, ez, mz;
};

// Calls f(bin, seg) for every piece of a particle's stencil.  The x-tile is
// the one holding the particle's home cell c_x (tiles are staged with an
// x-halo wide enough for the whole x-window); the y and z windows
// [jlo, jlo + nw - 1] are cut at tile boundaries and periodic images.
// bin = tile * 32 + (x0 mod 32), x0 the first node of the x-window in the
// tile's staged row: the tile kernels give bucket l to lane l.
template <typename F>
__device__ __forceinline__ void for_each_piece(const erpp_kparams& kp, int cx, const int jlo[3],
                                               const int nw[3], F f) {
  PieceSeg sg;
  sg.tx = cx / kp.T[0];
  const int bucket = (jlo[0] - sg.tx * kp.T[0] + kp.xhlo) & 31;
  const int jhy = jlo[1] + nw[1] - 1, jhz = jlo[2] + nw[2] - 1;
  for (int jy = jlo[1]; jy <= jhy;) {
    sg.my = erpp_floordiv(jy, kp.n[1]);
    const int wy = jy - sg.my * kp.n[1];
    sg.ty = wy / kp.T[1];
    sg.jy = jy;
    sg.ey = min(min((sg.ty + 1) * kp.T[1], kp.n[1]) - wy + jy - 1, jhy);
    for (int jz = jlo[2]; jz <= jhz;) {
      sg.mz = erpp_floordiv(jz, kp.n[2]);
      const int wz = jz - sg.mz * kp.n[2];
      sg.tz = wz / kp.T[2];
      sg.jz = jz;
      sg.ez = min(min((sg.tz + 1) * kp.T[2], kp.n[2]) - wz + jz - 1, jhz);
      const int tile = (sg.tz * kp.nt[1] + sg.ty) * kp.nt[0] + sg.tx;
      f(tile * 32 + bucket, sg);
      jz = sg.ez + 1;
    }
    jy = sg.ey + 1;
  }
}

// Design 4: the y-tile is the one holding the particle's home cell (tiles are
// staged with a y-halo); the z-window is cut at tile boundaries and periodic
// images.  In x the home cell's tile holds the whole window (x-halo tiles), or,
// with kp.xclip, the x-window is cut at x-tile boundaries and periodic images
// too, so that every piece stays inside its tile's columns.  Calls
// f(tile, qa, lx, x0, jz, ez, z0) per piece: window positions [qa, qa + lx)
// in x starting at staged column x0, planes [jz, ez] (z0 the first plane in
// the tile).
template <typename F>
__device__ __forceinline__ void for_each_piece4(const erpp_kparams& kp, const int c[3],
                                                const int jlo[3], const int nw[3], F f) {
  const int ty = c[1] / kp.T[1];
  const int jhx = jlo[0] + nw[0] - 1, jhz = jlo[2] + nw[2] - 1;
  for (int jx = jlo[0]; jx <= jhx;) {
    int tx, qa, lx, x0, ex;
    if (kp.xclip) {
      const int mx = erpp_floordiv(jx, kp.n[0]);
      const int wx = jx - mx * kp.n[0];
      tx = wx / kp.T[0];
      ex = min(min((tx + 1) * kp.T[0], kp.n[0]) - wx + jx - 1, jhx);
      qa = jx - jlo[0];
      lx = ex - jx + 1;
      x0 = kp.xoff + wx - tx * kp.T[0];
    } else {
      tx = c[0] / kp.T[0];
      ex = jhx;
      qa = 0;
      lx = nw[0];
      x0 = jlo[0] - (tx * kp.T[0] - kp.xoff);
    }
    for (int jz = jlo[2]; jz <= jhz;) {
      const int mz = erpp_floordiv(jz, kp.n[2]);
      const int wz = jz - mz * kp.n[2];
      const int tz = wz / kp.T[2];
      const int ez = min(min((tz + 1) * kp.T[2], kp.n[2]) - wz + jz - 1, jhz);
      f((tz * kp.nt[1] + ty) * kp.nt[0] + tx, qa, lx, x0, jz, ez, wz - tz * kp.T[2]);
      jz = ez + 1;
    }
    jx = ex + 1;
  }
}

// Geometry of particle i < n and its pieces' bins (the body of the count
// kernels): on_piece(k, bin) takes the particle's k-th piece a place in its
// bin.
template <typename OnPiece>
__device__ __forceinline__ void bin_count_one(
    const erpp_kparams& kp, int64_t i, int64_t n, const double* __restrict__ x0,
    const double* __restrict__ x1, const double* __restrict__ x2, float4* __restrict__ geo_t,
    int4* __restrict__ geo_c, float* __restrict__ xw, int xw_len, float* __restrict__ d0x,
    float4* __restrict__ lapc, float* __restrict__ up_acc, int64_t acc_stride, int ms,
    uint32_t* err, OnPiece on_piece) {
  double xv[3] = {x0[i], x1[i], x2[i]};
  if (up_acc && kp.design != 4) {
    up_acc[i] = 0.f;
    up_acc[acc_stride + i] = 0.f;
    up_acc[2 * acc_stride + i] = 0.f;
  }
  // 0 <= x < L on the bit patterns (non-negative doubles order as
  // integers; -0 is in range, NaN is not)
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(xv[a]);
    ok = ok && (bits < (unsigned long long)__double_as_longlong(kp.L[a]) || (bits << 1) == 0ull);
  }
  int c[3], off[3], nw[3], jlo[3];
  float t[3];
  if (ok) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // the window of erpp_axis_window (one FP64 product, the rest exact
      // integer and FP32 work)
      const erpp_axis_win aw =
          erpp_axis_window_lean(xv[a], kp.inv_dx[a], kp.cp[a], kp.cp_int[a], kp.cp_frac[a]);
      int ci = aw.ci;
      off[a] = aw.lo - ci;
      nw[a] = aw.hi - aw.lo + 1;
      t[a] = aw.t;
      // s can round up to exactly N for x just below L: the cell is then the
      // first one of the next image, which is the same node set shifted by N.
      if (ci >= kp.n[a]) ci -= kp.n[a];
      c[a] = ci;
      jlo[a] = ci + off[a];
    }
    bool inb = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      inb = inb && off[a] >= -kp.hlo && off[a] <= 0 && nw[a] >= 1 && nw[a] <= kp.xs;
    inb = inb && nw[0] <= xw_len;
    if (!inb) erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
    ok = inb;
  } else {
    erpp_set_err(err, ERPP_ERRBIT_RANGE);
  }
  // x-halo tiles: the particle's x-weights; x/y-halo tiles: the distance of
  // its x-window's first node, from which the tile kernels form the weights
  // (one of xw, d0x is null)
  float4* xw4 = xw ? reinterpret_cast<float4*>(xw + (size_t)i * xw_len) : nullptr;
  if (!ok) {
    if (d0x) d0x[i] = 0.f;
    if (lapc) {
      lapc[2 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
      lapc[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    geo_t[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    geo_c[i] = make_int4(0, 0, 0, 0);
    for (int k = 0; xw4 && k < xw_len / 4; ++k) xw4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  uint32_t pack = ERPP_GEO_VALID;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    pack |= (uint32_t)(-off[a]) << (4 * a);
    pack |= (uint32_t)nw[a] << (12 + 5 * a);
  }
  geo_c[i] = make_int4(c[0], c[1], c[2], (int)pack);
  const float d0 = (float)off[0] - t[0];
  if (d0x) d0x[i] = d0;
  if (lapc) {
    // the general force: the window's weight moments for the Laplacian
    float4 m[2];
    erpp_lap_moments(kp, t, off, nw, m);
    lapc[2 * i] = m[0];
    lapc[2 * i + 1] = m[1];
  }
  for (int k = 0; xw4 && k < xw_len / 4; ++k) {
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = 4 * k + j;
      const float d = d0 + (float)q;
      v[j] = q < nw[0] ? exp2f(-kp.beta[0] * d * d) : 0.f;
    }
    xw4[k] = make_float4(v[0], v[1], v[2], v[3]);
  }
  int k = 0;
  auto place = [&](int bin) {
    on_piece(k, bin);
    ++k;
  };
  if (kp.design == 4)
    for_each_piece4(kp, c, jlo, nw, [&](int tile, int, int, int, int, int, int) { place(tile); });
  else
    for_each_piece(kp, c[0], jlo, nw, [&](int bin, const PieceSeg&) { place(bin); });
  geo_t[i] = make_float4(t[0], t[1], t[2], __int_as_float(min(k, ms)));
}

__global__ void k_bin_count(erpp_kparams kp, int64_t n, const double* __restrict__ x0,
                            const double* __restrict__ x1, const double* __restrict__ x2,
                            float4* __restrict__ geo_t, int4* __restrict__ geo_c,
                            float* __restrict__ xw, int xw_len, float* __restrict__ d0x,
                            float4* __restrict__ lapc, float* __restrict__ up_acc,
                            int64_t acc_stride,
                            int32_t* __restrict__ tile_cnt, int32_t* __restrict__ slot, int ms,
                            uint32_t* err) {
  erpp_pdl_enter();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bin_count_one(kp, i, n, x0, x1, x2, geo_t, geo_c, xw, xw_len, d0x, lapc, up_acc, acc_stride,
                ms, err, [&](int k, int bin) {
                  const int v = atomicAdd(&tile_cnt[bin], 1);
                  if (k < ms)
                    slot[(int64_t)k * n + i] = v;
                  else
                    erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
                });
}

// Counting through a block histogram, for x/y-halo tiles with at most
// kHistBins tiles (small boxes, where many pieces fall into few tiles and the
// global increments of the counts would be contended): every piece of the
// block's 256 particles first takes a place in the block's shared count of
// its tile, each tile the block touches then takes the block's whole count
// from its global count in one increment, and a piece's place is that base
// plus its place in the block.  Called by the whole block (i >= n: no
// particle).  Pieces beyond kHistPieces of a particle are refused (bounds
// error); the caller uses it only when ms <= kHistPieces.
constexpr int kHistBins = 4096;
constexpr int kHistPieces = 24;

__device__ __forceinline__ void bin_count_hist(
    const erpp_kparams& kp, int64_t i, int64_t n, const double* __restrict__ x0,
    const double* __restrict__ x1, const double* __restrict__ x2, float4* __restrict__ geo_t,
    int4* __restrict__ geo_c, float* __restrict__ d0x, float4* __restrict__ lapc,
    int32_t* __restrict__ tile_cnt, int32_t* __restrict__ slot, int ms, int nbins,
    uint32_t* err, int32_t* hist) {
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  int bins[kHistPieces], loc[kHistPieces];
  int np = 0;
  if (i < n)
    bin_count_one(kp, i, n, x0, x1, x2, geo_t, geo_c, nullptr, kp.xs, d0x, lapc, nullptr, 0, ms,
                  err, [&](int k, int bin) {
                    if (k < ms && k < kHistPieces) {
                      bins[k] = bin;
                      loc[k] = atomicAdd(&hist[bin], 1);
                      np = k + 1;
                    } else {
                      erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
                    }
                  });
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    const int c = hist[b];
    if (c > 0) hist[b] = atomicAdd(&tile_cnt[b], c);
  }
  __syncthreads();
  for (int k = 0; k < np; ++k) slot[(int64_t)k * n + i] = hist[bins[k]] + loc[k];
}

__global__ void __launch_bounds__(256) k_bin_count_hist(
    erpp_kparams kp, int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
    const double* __restrict__ x2, float4* __restrict__ geo_t, int4* __restrict__ geo_c,
    float* __restrict__ d0x, float4* __restrict__ lapc, int32_t* __restrict__ tile_cnt,
    int32_t* __restrict__ slot, int ms, int nbins, uint32_t* err) {
  __shared__ int32_t hist[kHistBins];
  erpp_pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bin_count_hist(kp, i, n, x0, x1, x2, geo_t, geo_c, d0x, lapc, tile_cnt, slot, ms, nbins, err,
                 hist);
}

// Writes one record per piece, at its bin's start plus the place the piece
// took in k_bin_count (pieces visited in the same order); x/y-halo tiles keep
// that record position in slot[k][i] for the gather's per-piece sums.
__device__ __forceinline__ void bin_fill_one(const erpp_kparams& kp, int64_t i, int64_t n,
                                             const float4* __restrict__ geo_t,
                                             const int4* __restrict__ geo_c,
                                             const int32_t* __restrict__ start,
                                             int32_t* __restrict__ slot, int ms,
                                             int4* __restrict__ entries, int64_t cap,
                                             uint32_t* err) {
  const int4 g = geo_c[i];
  const uint32_t pack = (uint32_t)g.w;
  if (!(pack & ERPP_GEO_VALID)) return;
  const float4 gt = geo_t[i];
  const int c[3] = {g.x, g.y, g.z};
  int jlo[3], nw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    jlo[a] = c[a] + erpp_geo_off(pack, a);
    nw[a] = erpp_geo_nw(pack, a);
  }
  int k = 0;
  // x/y-halo tiles: each piece's place replaces its place in its bin, for the
  // gather's per-piece sums
  auto place = [&](int bin) -> int64_t {
    int64_t pos = cap;
    if (k < ms) {
      pos = (int64_t)start[bin] + slot[(int64_t)k * n + i];
      if (kp.design == 4) slot[(int64_t)k * n + i] = pos < cap ? (int32_t)pos : 0;
    }
    ++k;
    return pos;
  };
  if (kp.design == 4) {
    // record: {p, x0 | y0 << 7 | z0 << 13 | lz << 15 | qa << 18 | lx << 22 |
    //          ly << 27, d0y bits, d0z bits}: x0, y0 the staged x/y index of
    // the piece's first node, z0 its first plane in the tile, lz the planes in
    // the tile, [qa, qa + lx) the piece's positions in the particle's
    // x-window, ly the y-window length, d0 distances (grid units) of the first
    // y node / first plane
    const int ty = c[1] / kp.T[1];
    const int y0 = jlo[1] - (ty * kp.T[1] - kp.yhlo);
    const float d0y = (float)(jlo[1] - c[1]) - gt.y;
    const uint32_t fixed = ((uint32_t)y0 << 7) | ((uint32_t)nw[1] << 27);
    for_each_piece4(kp, c, jlo, nw, [&](int tile, int qa, int lx, int x0, int jz, int ez, int z0) {
      const float d0z = (float)(jz - c[2]) - gt.z;
      const uint32_t pk = fixed | (uint32_t)x0 | ((uint32_t)z0 << 13) |
                          ((uint32_t)(ez - jz + 1) << 15) | ((uint32_t)qa << 18) |
                          ((uint32_t)lx << 22);
      const int64_t pos = place(tile);
      if (pos < cap)
        entries[pos] = make_int4((int)i, (int)pk, __float_as_int(d0y), __float_as_int(d0z));
      else
        erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
    });
    return;
  }
  for_each_piece(kp, c[0], jlo, nw, [&](int bin, const PieceSeg& sg) {
    const int by = sg.ty * kp.T[1], bz = sg.tz * kp.T[2];
    const int x0 = jlo[0] - (sg.tx * kp.T[0] - kp.xhlo);
    const int l0y = sg.jy - sg.my * kp.n[1] - by;
    const int l0z = sg.jz - sg.mz * kp.n[2] - bz;
    const int base = l0z * kp.pxy + l0y * kp.px + x0;
    const int ly = sg.ey - sg.jy + 1, lz = sg.ez - sg.jz + 1;
    const float d0y = (float)(sg.jy - c[1]) - gt.y;
    const float d0z = (float)(sg.jz - c[2]) - gt.z;
    const int64_t pos = place(bin);
    if (pos < cap)
      entries[pos] = make_int4((int)i, base | (nw[0] << 17) | (ly << 22) | (lz << 27),
                               __float_as_int(d0y), __float_as_int(d0z));
    else
      erpp_set_err(err, ERPP_ERRBIT_BOUNDS);
  });
}

__global__ void k_bin_fill(erpp_kparams kp, int64_t n, const float4* __restrict__ geo_t,
                           const int4* __restrict__ geo_c, const int32_t* __restrict__ start,
                           int32_t* __restrict__ slot, int ms,
                           int4* __restrict__ entries, int64_t cap, uint32_t* err) {
  erpp_pdl_enter();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bin_fill_one(kp, i, n, geo_t, geo_c, start, slot, ms, entries, cap, err);
}

// Exclusive scan of the per-bin counts: k_scan_local scans chunks of
// kScanChunk bins (one block each) and writes the chunk totals, k_scan_top
// scans the totals in one block, k_scan_add offsets every chunk.
constexpr int kScanChunk = 4096;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_sums,
                                                        int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t ws = lane < nw ? warp_sums[lane] : 0;
    int32_t wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    warp_sums[lane] = wi - ws;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  int32_t r = warp_sums[warp] + incl - v;
  __syncthreads();
  return r;
}

// 1024 threads x 4 bins per thread = one chunk.
__global__ void k_scan_local(const int32_t* __restrict__ cnt, int32_t* __restrict__ start,
                             int32_t* __restrict__ chunk_tot, int nbins) {
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  const int base = blockIdx.x * kScanChunk + threadIdx.x * 4;
  int32_t v[4];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < nbins) ? cnt[base + k] : 0;
    s += v[k];
  }
  int32_t run = block_exclusive_scan(s, ws, &tot);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < nbins) start[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) chunk_tot[blockIdx.x] = tot;
}

__global__ void k_scan_top(int32_t* __restrict__ chunk_tot, int nchunks, int32_t* __restrict__ start,
                           int nbins) {
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  int32_t carry = 0;
  for (int c0 = 0; c0 < nchunks; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    const int32_t v = c < nchunks ? chunk_tot[c] : 0;
    const int32_t ex = block_exclusive_scan(v, ws, &tot);
    if (c < nchunks) chunk_tot[c] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[nbins] = carry;
}

__global__ void k_scan_add(int32_t* __restrict__ start, const int32_t* __restrict__ chunk_off,
                           int nbins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbins) return;
  start[i] += chunk_off[i / kScanChunk];
}

// ---- many boxes in one launch (batched boxes) ----
// Block b clears the counts of box b.
__global__ void k_zero_counts_multi(const erpp_box_dev* __restrict__ boxes) {
  const erpp_box_dev& B = boxes[blockIdx.x];
  for (int k = threadIdx.x; k < B.nbins; k += blockDim.x) B.tile_cnt[k] = 0;
}

// One block per (box, first particle) item of 256 particles.
__global__ void __launch_bounds__(256) k_bin_count_multi(const erpp_box_dev* __restrict__ boxes,
                                                         const int2* __restrict__ items) {
  __shared__ int32_t hist[kHistBins];
  const int2 it = items[blockIdx.x];
  const erpp_box_dev& B = boxes[it.x];
  const int64_t i = (int64_t)it.y + threadIdx.x;
  if (B.nbins <= kHistBins && B.ms <= kHistPieces) {  // the whole block
    bin_count_hist(B.kp, i, B.n, B.x[0], B.x[1], B.x[2], B.geo_t, B.geo_c, B.d0x, nullptr,
                   B.tile_cnt, B.piece_slot, B.ms, B.nbins, B.err, hist);
    return;
  }
  if (i >= B.n) return;
  bin_count_one(B.kp, i, B.n, B.x[0], B.x[1], B.x[2], B.geo_t, B.geo_c, nullptr, B.xw_len,
                B.d0x, nullptr, nullptr, B.cap, B.ms, B.err, [&](int k, int bin) {
                  const int v = atomicAdd(&B.tile_cnt[bin], 1);
                  if (k < B.ms)
                    B.piece_slot[(int64_t)k * B.n + i] = v;
                  else
                    erpp_set_err(B.err, ERPP_ERRBIT_BOUNDS);
                });
}

// One block of 1024 threads scans nbins counts into their starts (chunks of
// 4096 bins, the running total carried from chunk to chunk), total at
// start[nbins].
__device__ __forceinline__ void block_scan_bins(const int32_t* __restrict__ cnt,
                                                int32_t* __restrict__ start, int nbins) {
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  int32_t carry = 0;
  for (int c0 = 0; c0 < nbins; c0 += kScanChunk) {
    const int base = c0 + threadIdx.x * 4;
    int32_t v[4];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = (base + k < nbins) ? cnt[base + k] : 0;
      s += v[k];
    }
    int32_t run = carry + block_exclusive_scan(s, ws, &tot);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (base + k < nbins) start[base + k] = run;
      run += v[k];
    }
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[nbins] = carry;
}

// The scan of a box with at most kScanOneBins bins: one launch instead of
// three.  Up to 16384 bins each of the 1024 threads loads its run of 16
// counts at once (four 16-byte loads), so the block waits for one round trip;
// larger boxes go chunk by chunk.
constexpr int kScanOneBins = 65536;
__global__ void __launch_bounds__(1024) k_scan_one(const int32_t* __restrict__ cnt,
                                                   int32_t* __restrict__ start, int nbins) {
  erpp_pdl_enter();
  if (nbins > 16 * 1024 || (nbins & 15) != 0) {
    block_scan_bins(cnt, start, nbins);
    return;
  }
  __shared__ int32_t ws[32];
  __shared__ int32_t tot;
  const int base = threadIdx.x * 16;
  int4 v[4];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = base < nbins ? reinterpret_cast<const int4*>(cnt + base)[k] : make_int4(0, 0, 0, 0);
    s += v[k].x + v[k].y + v[k].z + v[k].w;
  }
  int32_t run = block_exclusive_scan(s, ws, &tot);
  if (base < nbins) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int4 o;
      o.x = run;
      o.y = o.x + v[k].x;
      o.z = o.y + v[k].y;
      o.w = o.z + v[k].z;
      run = o.w + v[k].w;
      reinterpret_cast<int4*>(start + base)[k] = o;
    }
  }
  if (threadIdx.x == 0) start[nbins] = tot;
}

// Block b scans the counts of box b into its starts.
__global__ void __launch_bounds__(1024) k_scan_multi(const erpp_box_dev* __restrict__ boxes) {
  const erpp_box_dev& B = boxes[blockIdx.x];
  block_scan_bins(B.tile_cnt, B.tile_start, B.nbins);
}

__global__ void __launch_bounds__(256) k_bin_fill_multi(const erpp_box_dev* __restrict__ boxes,
                                                        const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const erpp_box_dev& B = boxes[it.x];
  const int64_t i = (int64_t)it.y + threadIdx.x;
  if (i >= B.n) return;
  bin_fill_one(B.kp, i, B.n, B.geo_t, B.geo_c, B.tile_start, B.piece_slot, B.ms, B.entries,
               B.ecap, B.err);
}

}  // namespace

namespace erpp {

cudaError_t launch_scan(erpp_ctx* ctx, const int32_t* cnt, int32_t* start, int32_t* tmp,
                        int nbins, cudaStream_t st) {
  const int nchunks = (nbins + kScanChunk - 1) / kScanChunk;
  ctx->launches += 3;
  k_scan_local<<<nchunks, 1024, 0, st>>>(cnt, start, tmp, nbins);
  k_scan_top<<<1, 1024, 0, st>>>(tmp, nchunks, start, nbins);
  k_scan_add<<<(nbins + 255) / 256, 256, 0, st>>>(start, tmp, nbins);
  return cudaGetLastError();
}

cudaError_t bin_particles(erpp_ctx* ctx, int64_t n, const double* const x[3], bool zero_acc,
                          cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  const int nbins = erpp::nbins(kp);
  const int ms = ctx->maxseg[0] * ctx->maxseg[1] * ctx->maxseg[2];
  cudaError_t e = cudaMemsetAsync(ctx->tile_cnt, 0, sizeof(int32_t) * nbins, st);
  if (e != cudaSuccess) return e;
  if (n > 0 && kp.design == 4 && !kp.full_force && nbins <= kHistBins && ms <= kHistPieces) {
    // few tiles (a small box): count through block histograms
    ++ctx->launches;
    float4* no_lapc = nullptr;
    e = erpp_launch_pdl(k_bin_count_hist, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st,
                        0u, kp, n, x[0], x[1], x[2], ctx->geo_t, ctx->geo_c, ctx->d0x, no_lapc,
                        ctx->tile_cnt, ctx->piece_slot, ms, nbins, ctx->err);
    if (e != cudaSuccess) return e;
  } else if (n > 0) {
    int blocks = (int)((n + 255) / 256);
    ++ctx->launches;
    float* xw = kp.design == 4 ? nullptr : ctx->xw;
    float* d0x = kp.design == 4 ? ctx->d0x : nullptr;
    float4* lapc = kp.design == 4 && kp.full_force ? ctx->lapc : nullptr;
    float* up_acc = zero_acc ? ctx->up_acc : nullptr;
    e = erpp_launch_pdl(k_bin_count, dim3(blocks), dim3(256), 0, st, 0u, kp, n, x[0], x[1], x[2],
                        ctx->geo_t, ctx->geo_c, xw, ctx->xw_len, d0x, lapc, up_acc, ctx->cap,
                        ctx->tile_cnt, ctx->piece_slot, ms, ctx->err);
    if (e != cudaSuccess) return e;
  }
  const int nchunks = (nbins + kScanChunk - 1) / kScanChunk;
  if (nbins <= kScanOneBins) {
    ++ctx->launches;
    e = erpp_launch_pdl(k_scan_one, dim3(1), dim3(1024), 0, st, 0u,
                        (const int32_t*)ctx->tile_cnt, ctx->tile_start, nbins);
    if (e != cudaSuccess) return e;
  } else {
    ctx->launches += 3;
    k_scan_local<<<nchunks, 1024, 0, st>>>(ctx->tile_cnt, ctx->tile_start, ctx->scan_tmp, nbins);
    k_scan_top<<<1, 1024, 0, st>>>(ctx->scan_tmp, nchunks, ctx->tile_start, nbins);
    k_scan_add<<<(nbins + 255) / 256, 256, 0, st>>>(ctx->tile_start, ctx->scan_tmp, nbins);
  }
  if (n > 0) {
    int blocks = (int)((n + 255) / 256);
    ++ctx->launches;
    e = erpp_launch_pdl(k_bin_fill, dim3(blocks), dim3(256), 0, st, 0u, kp, n,
                        (const float4*)ctx->geo_t, (const int4*)ctx->geo_c,
                        (const int32_t*)ctx->tile_start, ctx->piece_slot, ms, ctx->entries,
                        ctx->entries_cap, ctx->err);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}


cudaError_t launch_bin_multi(const erpp_box_dev* boxes, int nbox, const int2* pitems,
                             int npitems, cudaStream_t st) {
  k_zero_counts_multi<<<nbox, 256, 0, st>>>(boxes);
  if (npitems > 0) k_bin_count_multi<<<npitems, 256, 0, st>>>(boxes, pitems);
  k_scan_multi<<<nbox, 1024, 0, st>>>(boxes);
  if (npitems > 0) k_bin_fill_multi<<<npitems, 256, 0, st>>>(boxes, pitems);
  return cudaGetLastError();
}

}  // namespace erpp
