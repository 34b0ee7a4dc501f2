// erpp_tiles4.cu -- FP32 tile kernels with lockstep unit schedules: the
// kernel gather and the regularised source scatter (Sec. 2.4, Eq.
// ns_regularized_filtered; the heat kernel of App. A.1 factored per axis).
//
// Tiles.  A thread block owns a tile of W x T_y x T_z nodes and stages it in
// shared memory with an x-halo (xhlo below, xhhi above) and a y-halo (yhlo,
// yhhi): every particle whose home cell lies in the tile's x/y range finds its
// whole x- and y-window there, so a particle's stencil is cut only along z
// (one "piece" per z-tile it reaches).  Staged layout [3][T_z][NY][PX] with
// NY = T_y + yhlo + yhhi rows, PX floats per row and the tile's first column
// at x' = xoff (xhlo rounded up to a multiple of 4, so that the interior is
// 16-byte aligned); PX and the plane pitch PXY are both 16 (mod 32), so node
// (x', y', z') sits in shared-memory bank (x' + 16 (y' + z')) mod 32.
// Staging: a tile whose staged box needs no periodic wrap (and whose layout
// has no plane padding) is loaded by one TMA copy of the 4D box
// (x, y, z, component) of the field, completed on an mbarrier; a wrapping tile
// with 16-byte aligned rows by one bulk copy per staged row and periodic
// segment (same mbarrier); any other by 4-byte asynchronous copies.  Each
// thread's record of the first batch is loaded before the staging is issued,
// so that the two latencies overlap.
//
// Units and buckets.  A unit is one z-plane of a piece: ly rows of lx nodes,
// the same for every particle (lx, ly = the window lengths).  Walking its rows
// one per step, a unit's first node moves by 16 banks per row, in step with
// every other unit walked at the same time, so each unit has a fixed bucket
//   b = (x0 + 16 (first row + z)) mod 32
// relative to the others: 32 units with 32 different buckets, processed row
// by row in lockstep by the 32 lanes of a warp, never share a bank.  A unit
// may start at its second row and end with its first (a rotation of its
// rows), which moves it to bucket b ^ 16 (for an even ly without any cost; for
// an odd ly its last row may share a bank); the schedule splits the units of
// every bucket pair evenly between its two buckets.
//
// Schedule.  Per batch of pieces (at most one per thread) the block builds a
// table sched[round][warp][lane]: bucket b's k-th unit goes to lane b of warp
// k mod NW in round k / NW (NW warps per block), for the fewest rounds R that
// hold every unit; units beyond a bucket's NW R slots fill the free slots of
// other buckets, last rounds first (those lanes then share banks with the
// slot's own bucket).  Every warp runs its R rounds
// independently; in a round all lanes walk their units' rows together (the
// longest window of the round), so a unit switch is a few shared-memory reads
// per lane.  The batch's piece records and x-weights are staged in shared
// memory with the schedule.
//
// Weights are separable, w = e_x(q) * 2^(-(beta_y d_y^2 + beta_z d_z^2)) with
// e_x the particle's x-weights (precomputed by the binning), d in grid units.
//
// Gather: a lane sums w*u over its unit and stores the three totals in the
// unit's own (piece, plane) slot; the block adds each piece's planes in
// plane order and stores the sums at the place of the piece's record, and the
// particle adds its pieces in piece order afterwards (no atomics, so the
// gathered velocity is reproducible bit for bit).
//
// Scatter: 32-bit fixed point with shared-memory integer atomics (order
// independent), per-tile scale 2^30 / B with B = sum over the tile's pieces of
// max|f| (no sum can overflow).  Per unit G = round(f e_x e_z 2^30 / B) per
// component and x-slot, per row W = round(e_y 2^31), and each node receives
// the high word of G W + 2^31 (one wide multiply-add and one atomic per node
// component).  A tile of one batch sums B from its staged forces, a larger
// one by a pass over its entries first.  Tiles with more than 1024 pieces add
// FP32 values instead.  ERPP_KAHAN (the compensated mode) keeps 47 bits of
// every exact 64-bit product G W (scale 2^31 / B, one bit finer) in two
// 32-bit sums per node, the high words and the top bits of the low words: no
// rounding of the sums, a truncation of each product far below the
// rounding of its factors.  Tiles of 65536 pieces or more add FP32 values.  The final values are formed in shared memory and every staged row
// leaves by one bulk asynchronous copy (interior rows to S, y-halo rows to a
// strip buffer), the x-halo columns by plain stores; k_merge_rows and
// k_merge_cols then add the strips to the neighbouring tiles in a fixed
// order.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "erpp_internal.cuh"

namespace {

// Threads per block of the tile kernels: 256 or 512 (a tiling option).
constexpr int kDenseTile = 1024;  // pieces above which a tile accumulates in FP32
constexpr int kSplitMaxPieces = 65535;  // compensated mode: most pieces of a split-word tile
constexpr uint16_t kEmpty = 0xffffu;

// Pieces per batch: smaller batches for the 16-float x-weight records keep
// two blocks per SM.
template <int XW>
struct Batch {
  // (the gather may take batches twice as large: gather_big_batch)
  static constexpr int kPB = XW <= 8 ? 256 : 128;
};

// Piece record (from the binning): p, packed geometry, d0y, d0z (distances,
// in grid units, from the particle to the first node of its y-window and to
// the piece's first plane).  The piece covers positions [qa, qa + lx) of the
// particle's x-window (qa > 0 or a shorter lx only when the window is cut at
// x-tile boundaries).
struct Piece4 {
  int p;
  int x0, y0, z0, lz, qa, lx, ly;
  float d0y, d0z;
};

__device__ __forceinline__ Piece4 unpack4(int4 r) {
  Piece4 pc;
  pc.p = r.x;
  const uint32_t v = (uint32_t)r.y;
  pc.x0 = (int)(v & 127u);
  pc.y0 = (int)((v >> 7) & 63u);
  pc.z0 = (int)((v >> 13) & 3u);
  pc.lz = (int)((v >> 15) & 7u);
  pc.qa = (int)((v >> 18) & 15u);
  pc.lx = (int)((v >> 22) & 31u);
  pc.ly = (int)(v >> 27);
  pc.d0y = __int_as_float(r.z);
  pc.d0z = __int_as_float(r.w);
  return pc;
}

// The x-weights of a unit: 2^(-beta_x d^2) at its slots q (window position
// qa + q, distance d0x + qa + q with d0x that of the window's first node),
// 0 past the piece's lx slots.  The binning's normalisation takes the same
// values with the same arithmetic.
template <int XM>
__device__ __forceinline__ void make_ex(const Piece4& pc, float d0x, float bx, float (&ex)[XM]) {
#pragma unroll
  for (int q = 0; q < XM; ++q) {
    const float d = d0x + (float)(pc.qa + q);
    ex[q] = q < pc.lx ? exp2f(-bx * d * d) : 0.f;
  }
}

// ---- asynchronous global -> shared copies (cp.async) ----
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
// Shared-memory writes of this thread made visible to the asynchronous proxy
// (bulk copies issued after the next barrier read them).
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Bulk copy shared -> global (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_store_s2g(void* dst, unsigned src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
               :: "l"(dst), "r"(src), "r"(bytes) : "memory");
}
// Waits until this thread's bulk copies have read their shared-memory source.
__device__ __forceinline__ void bulk_commit_wait_read() {
  asm volatile("cp.async.bulk.commit_group;\n\tcp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

// ---- TMA box load completed on an mbarrier (bounded wait) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Before the barrier's memory is initialised again (a persistent block that
// stages one tile after another).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Waits for phase `parity` of the barrier for at most `limit_ns` nanoseconds
// (the global timer); false when the phase has not completed by then.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, unsigned parity, int64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((int64_t)(globaltimer_ns() - t0) > limit_ns) return false;
  }
}
// Bulk copy global -> shared completed on an mbarrier (both 16-byte aligned,
// bytes a multiple of 16).
__device__ __forceinline__ void bulk_load_g2s(unsigned dst, const void* src, unsigned bytes,
                                              unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// ---- thread-block clusters: rank, barrier, distributed shared memory ----
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
// Every thread of every block of the cluster arrives (release: this block's
// earlier memory accesses are ordered before the others' waits return).
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// The address of the same shared-memory location in block `rank` of the cluster.
__device__ __forceinline__ unsigned mapa_shared(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_cluster_f32(unsigned addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

// ---- shared-memory accesses by 32-bit shared address, immediate offsets ----
__device__ __forceinline__ unsigned shared_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
template <int OFF>
__device__ __forceinline__ float lds_f32(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];\n" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void red_s32(unsigned a, int v) {
  asm volatile("red.shared.add.s32 [%0+%1], %2;\n" ::"r"(a), "n"(OFF), "r"(v));
}
template <int OFF>
__device__ __forceinline__ void red_f32(unsigned a, float v) {
  asm volatile("red.shared.add.f32 [%0+%1], %2;\n" ::"r"(a), "n"(OFF), "f"(v));
}

// round(g w / 2^32) = high word of g w + 2^31: the low word of the product
// plus 2^31 (carry out), then the signed high word plus that carry.
__device__ __forceinline__ int mul_hi_round(int g, int w) {
  int hi;
  asm("{\n\t.reg .u32 lo;\n\t"
      "mad.lo.cc.u32 lo, %1, %2, 0x80000000;\n\t"
      "madc.hi.s32 %0, %1, %2, 0;\n\t}\n"
      : "=r"(hi)
      : "r"(g), "r"(w));
  return hi;
}

// One row of a unit, slot Q onwards.  Gather: x_c += e_x(q) u_c(q) over the
// row (the weights of slots past the piece are 0, and every word a slot can
// reach holds a finite value: staged field, or zeros the gather wrote).
// Scatter (fixed point): u_c(q) += high word of G_c(q) W.  Scatter (FP32):
// u_c(q) += f_c w e_x(q).  a0..a2: shared addresses of the row's first node
// per component.  Slots Q < NQ are visited (NQ = LMIN when no lane's window
// is longer: slots past a window have weight 0 and add nothing).
template <int Q, int XM, int NQ = XM>
__device__ __forceinline__ void row_dot(unsigned a0, unsigned a1, unsigned a2, const float (&ex)[XM],
                                        float& x0, float& x1, float& x2) {
  if constexpr (Q < NQ) {
    x0 = fmaf(ex[Q], lds_f32<4 * Q>(a0), x0);
    x1 = fmaf(ex[Q], lds_f32<4 * Q>(a1), x1);
    x2 = fmaf(ex[Q], lds_f32<4 * Q>(a2), x2);
    row_dot<Q + 1, XM, NQ>(a0, a1, a2, ex, x0, x1, x2);
  }
}

// row_dot with a second set of x-weights on the same loaded values: x_c +=
// e_x(q) u_c(q) and y_c += e2_x(q) u_c(q) (the general force's gather of the
// velocity and of its Laplacian).
template <int Q, int XM, int NQ = XM>
__device__ __forceinline__ void row_dot2(unsigned a0, unsigned a1, unsigned a2,
                                         const float (&ex)[XM], const float (&e2)[XM], float& x0,
                                         float& x1, float& x2, float& y0, float& y1, float& y2) {
  if constexpr (Q < NQ) {
    const float u0 = lds_f32<4 * Q>(a0), u1 = lds_f32<4 * Q>(a1), u2 = lds_f32<4 * Q>(a2);
    x0 = fmaf(ex[Q], u0, x0);
    x1 = fmaf(ex[Q], u1, x1);
    x2 = fmaf(ex[Q], u2, x2);
    y0 = fmaf(e2[Q], u0, y0);
    y1 = fmaf(e2[Q], u1, y1);
    y2 = fmaf(e2[Q], u2, y2);
    row_dot2<Q + 1, XM, NQ>(a0, a1, a2, ex, e2, x0, x1, x2, y0, y1, y2);
  }
}

template <int Q, int XM, int LMIN, int NQ = XM>
__device__ __forceinline__ void row_red_fixed(unsigned a0, unsigned a1, unsigned a2,
                                              const int (&G0)[XM], const int (&G1)[XM],
                                              const int (&G2)[XM], int W, int lx) {
  if constexpr (Q < NQ) {
    if (Q < LMIN || Q < lx) {
      red_s32<4 * Q>(a0, mul_hi_round(G0[Q], W));
      red_s32<4 * Q>(a1, mul_hi_round(G1[Q], W));
      red_s32<4 * Q>(a2, mul_hi_round(G2[Q], W));
    }
    row_red_fixed<Q + 1, XM, LMIN, NQ>(a0, a1, a2, G0, G1, G2, W, lx);
  }
}

template <int Q, int XM, int LMIN, int NQ = XM>
__device__ __forceinline__ void row_red_f32(unsigned a0, unsigned a1, unsigned a2,
                                            const float (&ex)[XM], float f0, float f1, float f2,
                                            float wy, int lx) {
  if constexpr (Q < NQ) {
    if (Q < LMIN || Q < lx) {
      const float wq = wy * ex[Q];
      red_f32<4 * Q>(a0, f0 * wq);
      red_f32<4 * Q>(a1, f1 * wq);
      red_f32<4 * Q>(a2, f2 * wq);
    }
    row_red_f32<Q + 1, XM, LMIN, NQ>(a0, a1, a2, ex, f0, f1, f2, wy, lx);
  }
}

// Compensated mode: the exact 64-bit product G_c(q) W = 2^32 H + L is added
// as two 32-bit fixed-point words, the signed high word H to the node's high
// sum and the top 15 bits of the low word L to its low sum (at offset lo):
// both are sums of at most one term per piece (H below 2^30 + 1, L >> 17
// below 2^15), which cannot overflow for fewer than 65536 pieces.
template <int OFF>
__device__ __forceinline__ void red_split(unsigned a, unsigned lo, int g, int w) {
  int h;
  unsigned l;
  asm("mul.hi.s32 %0, %2, %3;\n\tmul.lo.s32 %1, %2, %3;\n" : "=r"(h), "=r"(l) : "r"(g), "r"(w));
  red_s32<OFF>(a, h);
  red_s32<OFF>(a + lo, (int)(l >> 17));
}

template <int Q, int XM, int LMIN, int NQ = XM>
__device__ __forceinline__ void row_red_split(unsigned a0, unsigned a1, unsigned a2, unsigned lo,
                                              const int (&G0)[XM], const int (&G1)[XM],
                                              const int (&G2)[XM], int W, int lx) {
  if constexpr (Q < NQ) {
    if (Q < LMIN || Q < lx) {
      red_split<4 * Q>(a0, lo, G0[Q], W);
      red_split<4 * Q>(a1, lo, G1[Q], W);
      red_split<4 * Q>(a2, lo, G2[Q], W);
    }
    row_red_split<Q + 1, XM, LMIN, NQ>(a0, a1, a2, lo, G0, G1, G2, W, lx);
  }
}

// Dynamic shared memory of one block: the staged field (copies * plane
// floats), then the batch's records, force words (scatter), x-distances,
// Laplacian moments (general-force gather), unit words, schedule and piece
// accumulators (gather: value sums, and Laplacian sums with lap).
template <int PB>
struct Carve {
  float* field;
  int4* rec;
  float4* fsb;
  float* dxb;
  float4* lcb;
  uint32_t* unit;
  uint16_t* sched;
  float* pacc;
};

// Floats after the staged field that the gather keeps at zero: a unit's last
// slots may reach past the last staged row.
constexpr int kFieldPad = 16;

// The unit words, the schedule and the gather's piece accumulators are sized
// for the tile's tz planes (a piece has at most tz units); the schedule holds
// whole rounds of up to 512 threads.
template <int PB>
__host__ __device__ inline size_t carve_bytes(int plane, int tz, int copies, bool gather,
                                              bool lap = false) {
  const int NU = PB * tz, NS = (NU + 511) & ~511;
  size_t b = ((size_t)copies * plane + kFieldPad) * 4;
  b += (size_t)PB * 16;          // rec
  if (!gather) b += (size_t)PB * 16;  // fsb
  b += (size_t)PB * 4;           // dxb
  b = (b + 15) & ~(size_t)15;
  if (lap) b += (size_t)PB * 32;  // lcb
  b += (size_t)NU * 4;           // unit
  b += (size_t)NS * 2;           // sched
  b = (b + 15) & ~(size_t)15;
  if (gather) b += (size_t)(lap ? 6 : 3) * tz * PB * 4;  // pacc
  return b;
}

template <int PB>
__device__ inline Carve<PB> carve(unsigned char* base, int plane, int tz, int copies, bool gather,
                                  bool lap = false) {
  const int NU = PB * tz, NS = (NU + 511) & ~511;
  Carve<PB> c;
  size_t o = 0;
  c.field = reinterpret_cast<float*>(base);
  o += ((size_t)copies * plane + kFieldPad) * 4;
  c.rec = reinterpret_cast<int4*>(base + o);
  o += (size_t)PB * 16;
  c.fsb = reinterpret_cast<float4*>(base + o);
  if (!gather) o += (size_t)PB * 16;
  c.dxb = reinterpret_cast<float*>(base + o);
  o += (size_t)PB * 4;
  o = (o + 15) & ~(size_t)15;
  c.lcb = reinterpret_cast<float4*>(base + o);
  if (lap) o += (size_t)PB * 32;
  c.unit = reinterpret_cast<uint32_t*>(base + o);
  o += (size_t)NU * 4;
  c.sched = reinterpret_cast<uint16_t*>(base + o);
  o += (size_t)NS * 2;
  o = (o + 15) & ~(size_t)15;
  c.pacc = reinterpret_cast<float*>(base + o);
  return c;
}

struct SchedState {
  int pair[16];
  int cnt[32];
  int vpre[33];
  int nunits;
  int novf;
};

__device__ __forceinline__ void tile_origin4(const erpp_kparams& kp, int tile, int b[3],
                                             int ext[3], int t[3]) {
  const int txy = kp.nt[0] * kp.nt[1];
  t[2] = tile / txy;
  const int r = tile - t[2] * txy;
  t[1] = r / kp.nt[0];
  t[0] = r - t[1] * kp.nt[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b[a] = t[a] * kp.T[a];
    ext[a] = min(b[a] + kp.T[a], kp.n[a]) - b[a];
  }
}

// Issues the copies that stage the tile with its x/y halo (periodic wrap);
// the columns outside [xoff - xhlo, xoff + ext_x + xhhi) are set to zero.
template <int NT>
__device__ void stage_tile4(const erpp_kparams& kp, const float* __restrict__ u, float* field,
                            const int b[3], const int ext[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int ny_st = ext[1] + kp.yhlo + kp.yhhi;
  const int hx = kp.xhlo + kp.xhhi;
  // 16-byte chunks for the interior when rows and tile starts are aligned
  const bool vec = (kp.n[0] & 3) == 0 && (ext[0] & 3) == 0 && (b[0] & 3) == 0 &&
                   (((uintptr_t)u) & 15) == 0;
  const int nvec = vec ? ext[0] >> 2 : 0;
  const int nscal = (vec ? 0 : ext[0]) + hx;
  const int jobs = nvec + nscal;
  for (int c = 0; c < 3; ++c) {
    for (int z = 0; z < ext[2]; ++z) {
      const float* gplane = u + c * nn + (size_t)(b[2] + z) * kp.n[1] * kp.n[0];
      float* splane = field + c * kp.plane + z * kp.pxy;
      for (int y = warp; y < ny_st; y += NT / 32) {
        int gy = b[1] - kp.yhlo + y;
        gy = gy < 0 ? gy + kp.n[1] : (gy >= kp.n[1] ? gy - kp.n[1] : gy);
        const float* grow = gplane + (size_t)gy * kp.n[0];
        float* srow = splane + y * kp.px;
        // columns left of and right of the staged range: zeros
        const int clo = kp.xoff - kp.xhlo, chi = kp.xoff + ext[0] + kp.xhhi;
        for (int j = lane; j < clo + (kp.px - chi); j += 32) srow[j < clo ? j : chi + (j - clo)] = 0.f;
        for (int j = lane; j < jobs; j += 32) {
          if (j < nvec) {
            cp_async16(srow + kp.xoff + 4 * j, grow + b[0] + 4 * j);
          } else {
            const int s = j - nvec;  // scalar job: interior (non-vec) then halo
            int xl, gx;
            if (!vec && s < ext[0]) {
              xl = kp.xoff + s;
              gx = b[0] + s;
            } else {
              const int h = vec ? s : s - ext[0];
              if (h < kp.xhlo) {
                xl = kp.xoff - kp.xhlo + h;
                gx = b[0] - kp.xhlo + h;
              } else {
                xl = kp.xoff + ext[0] + (h - kp.xhlo);
                gx = b[0] + ext[0] + (h - kp.xhlo);
              }
              gx = gx < 0 ? gx + kp.n[0] : (gx >= kp.n[0] ? gx - kp.n[0] : gx);
            }
            cp_async4(srow + xl, grow + gx);
          }
        }
      }
    }
  }
}

// Bytes that stage_tile_rows copies for a tile: every staged row in full.
__device__ __forceinline__ unsigned tile_rows_bytes(const erpp_kparams& kp, const int ext[3]) {
  return 4u * (unsigned)(3 * ext[2] * (ext[1] + kp.yhlo + kp.yhhi) * kp.px);
}

// Stages the tile with its x/y halo by bulk copies, one per staged row and
// periodic segment of it (the rows' px columns start at x = b_x - xoff), all
// completing on `bar`, whose expected bytes are already set.  Needs rows of
// a multiple of 4 floats and a 16-byte aligned field.
template <int NT>
__device__ void stage_tile_rows(const erpp_kparams& kp, const float* __restrict__ u, float* field,
                                const int b[3], const int ext[3], uint64_t* bar) {
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int ny_st = ext[1] + kp.yhlo + kp.yhhi;
  const int nrow = 3 * ext[2] * ny_st;
  const unsigned fbase = smem_u32(field), mb = smem_u32(bar);
  int gx0 = (b[0] - kp.xoff) % kp.n[0];
  gx0 = gx0 < 0 ? gx0 + kp.n[0] : gx0;
  for (int r = threadIdx.x; r < nrow; r += NT) {
    const int cz = r / ny_st;
    const int y = r - cz * ny_st;
    const int cc = cz / ext[2];
    const int z = cz - cc * ext[2];
    int gy = b[1] - kp.yhlo + y;
    gy = gy < 0 ? gy + kp.n[1] : (gy >= kp.n[1] ? gy - kp.n[1] : gy);
    const float* grow = u + cc * nn + ((size_t)(b[2] + z) * kp.n[1] + gy) * kp.n[0];
    unsigned dst = fbase + 4u * (unsigned)(cc * kp.plane + z * kp.pxy + y * kp.px);
    int gx = gx0, left = kp.px;
    while (left > 0) {
      const int seg = min(left, kp.n[0] - gx);
      bulk_load_g2s(dst, grow + gx, 4u * (unsigned)seg, mb);
      dst += 4u * (unsigned)seg;
      left -= seg;
      gx = 0;
    }
  }
}

// Builds the unit schedule of pieces [0, np) (records in cv.rec).  Returns
// the number of rounds.  Called by the whole block; synchronises.
template <int PB, int NT>
__device__ int build_schedule(const Carve<PB>& cv, SchedState& ss, int np) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x;
  if (tid < 16) ss.pair[tid] = 0;
  if (tid == 0) {
    ss.nunits = 0;
    ss.novf = 0;
  }
  __syncthreads();
  // Buckets b and b ^ 16 form a pair (every unit can take either, by rotating
  // its rows): the k-th unit of a pair goes to the lower bucket for even k and
  // to the upper one for odd k, so a pair's units split evenly.
  for (int k = tid; k < np; k += NT) {
    const Piece4 pc = unpack4(cv.rec[k]);
    const int ub = atomicAdd(&ss.nunits, pc.lz);
    for (int z = 0; z < pc.lz; ++z) {
      const int natural = (pc.x0 + 16 * ((pc.y0 + pc.z0 + z) & 1)) & 31;
      const int pr = natural & 15;
      const int idx = atomicAdd(&ss.pair[pr], 1);
      const int bucket = pr + 16 * (idx & 1);
      const uint32_t rot = bucket != natural ? 1u : 0u;
      cv.unit[ub + z] = (uint32_t)k | ((uint32_t)z << 10) | ((uint32_t)bucket << 14) |
                        ((uint32_t)min(idx >> 1, 4095) << 19) | (rot << 31);
    }
  }
  __syncthreads();
  if (tid < 32) ss.cnt[tid] = (ss.pair[tid & 15] + (tid < 16 ? 1 : 0)) >> 1;
  // Rounds: the fewest that hold every unit (measured faster than one more
  // round that would leave no bucket overflowing)
  const int U = ss.nunits;
  const int R = (U + NT - 1) / NT;
  const int cap = NW * R;
  if (tid < 32) {
    const int vac = max(0, cap - ss.cnt[tid]);
    int incl = vac;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += t;
    }
    ss.vpre[tid + 1] = incl;
    if (tid == 0) ss.vpre[0] = 0;
  }
  for (int s = tid; s < R * NT; s += NT) cv.sched[s] = kEmpty;
  __syncthreads();
  for (int u = tid; u < U; u += NT) {
    const uint32_t w = cv.unit[u];
    int bucket = (int)((w >> 14) & 31u);
    int slot = (int)((w >> 19) & 4095u);
    if (slot >= cap) {
      // overflow: the v-th free slot, free slots of each bucket in order
      const int v = atomicAdd(&ss.novf, 1);
      int lo = 0, hi = 32;  // bucket with vpre[b] <= v < vpre[b + 1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ss.vpre[mid] <= v) lo = mid; else hi = mid;
      }
      bucket = lo;
      slot = cap - 1 - (v - ss.vpre[lo]);  // latest rounds first
    }
    cv.sched[(slot / NW) * NT + (slot % NW) * 32 + bucket] = (uint16_t)u;
  }
  __syncthreads();
  return R;
}

// Even split of a tile's pieces into batches of at most PB.
__device__ __forceinline__ int batch_size(int total, int PB) {
  const int nb = (total + PB - 1) / PB;
  return (total + nb - 1) / nb;
}

// Thread k loads record k of the batch (issued early, so that its latency
// overlaps other work), then stages it and, through the particle index, the
// particle's x-distance and (scatter) force word (asynchronous copies); a
// batch larger than the block stages its further records k + NT, ... too.
__device__ __forceinline__ int4 load_rec(const int4* __restrict__ entries, int b0, int np) {
  return threadIdx.x < np ? __ldg(&entries[b0 + threadIdx.x]) : make_int4(0, 0, 0, 0);
}
template <int PB, bool FORCES, bool LAP = false>
__device__ __forceinline__ void stage_one(const Carve<PB>& cv, int k, int4 r,
                                          const float* __restrict__ d0x,
                                          const float4* __restrict__ fscat,
                                          const float4* __restrict__ lapc) {
  cv.rec[k] = r;
  cp_async4(cv.dxb + k, d0x + r.x);
  if (FORCES) cp_async16(cv.fsb + k, fscat + r.x);
  if (LAP) {
    cp_async16(cv.lcb + 2 * k, lapc + 2 * (size_t)r.x);
    cp_async16(cv.lcb + 2 * k + 1, lapc + 2 * (size_t)r.x + 1);
  }
}
template <int PB, bool FORCES, bool LAP = false>
__device__ void stage_batch(const Carve<PB>& cv, int4 r, int np, int b0,
                            const int4* __restrict__ entries, const float* __restrict__ d0x,
                            const float4* __restrict__ fscat,
                            const float4* __restrict__ lapc = nullptr) {
  const int k = threadIdx.x;
  if (k < np) stage_one<PB, FORCES, LAP>(cv, k, r, d0x, fscat, lapc);
  if constexpr (PB > 256) {
    for (int j = k + blockDim.x; j < np; j += blockDim.x)
      stage_one<PB, FORCES, LAP>(cv, j, __ldg(&entries[b0 + j]), d0x, fscat, lapc);
  }
}

// One unit of a round: rows visited from row `rot` on, wrapping once.
struct UnitRows {
  int base;    // shared index of the unit's first node (row 0)
  int ly, lx;
  int rot;
  float d0y, ezz;
};

// The gather of one tile, called by the whole block (the body of k_gather4
// and of the multi-box gather).  XM: longest x-window; LMIN: shortest (slots
// q >= LMIN are tested); XW: 8 for windows of at most 7 nodes, else 16 (sets
// the pieces per batch).  LAP: also the Laplacian of the gathered velocity
// (general force, Eq. force_particle): per row, the same loaded values
// against the x-weights' second-derivative factors, and the row's and
// plane's own factors.  tmap: the field's tensor map (parameter or global
// memory).  Returns bit 0: a bounded wait ran out (the block gave the tile
// up); bit 1: the staging barriers were initialised.
template <int XM, int LMIN, int XW, int NT, bool LAP, int PB>
__device__ __forceinline__ int gather_tile4(
    const erpp_kparams& kp, int tile, const float* __restrict__ u, const CUtensorMap* tmap,
    int use_tma, const int32_t* __restrict__ start, const int4* __restrict__ entries,
    int64_t ecap, const float* __restrict__ d0x, const float4* __restrict__ lapc,
    float4* __restrict__ up_part, float4* __restrict__ lap_part, uint32_t* err,
    unsigned char* smem_raw, SchedState& ss, uint64_t& tma_bar, uint64_t& stall_bar) {
  static_assert(PB <= 1024, "unit words hold the piece index in 10 bits");
  const int e0 = start[tile];
  const int e1 = (int)min((int64_t)start[tile + 1], ecap);
  if (e0 >= e1) return 0;
  const int tzs = kp.T[2];  // planes per tile: units per piece, at most
  const Carve<PB> cv = carve<PB>(smem_raw, kp.plane, tzs, 3, true, LAP);
  int b[3], ext[3], tt[3];
  tile_origin4(kp, tile, b, ext, tt);
  // one TMA box when the staged rows need no periodic wrap
  const int hy = kp.yhlo + kp.yhhi;
  const int x0 = b[0] - kp.xoff, y0 = b[1] - kp.yhlo;
  const bool tma = use_tma && x0 >= 0 && x0 + kp.px <= kp.n[0] && y0 >= 0 &&
                   y0 + kp.T[1] + hy <= kp.n[1];
  const int bs = batch_size(e1 - e0, PB);
  const int4 rfirst = load_rec(entries, e0, min(bs, e1 - e0));
  // otherwise bulk row copies when rows are whole 16-byte chunks, else
  // word-level asynchronous copies
  const bool rows = !tma && (kp.n[0] & 3) == 0 && (b[0] & 3) == 0 && (kp.xoff & 3) == 0 &&
                    (kp.px & 3) == 0 && (((uintptr_t)u) & 15) == 0;
  if (threadIdx.x == 0 && (tma || rows)) {
    mbar_init(&tma_bar, 1);
    if (kp.debug_stall) mbar_init(&stall_bar, 1);
    if (tma) {
      mbar_expect_tx(&tma_bar, (unsigned)(3 * kp.plane * 4));
      tma_load_4d(cv.field, tmap, &tma_bar, x0, y0, b[2], 0);
    } else {
      mbar_expect_tx(&tma_bar, tile_rows_bytes(kp, ext));
    }
  }
  if (rows) {
    __syncthreads();  // the barrier is initialised and expects the bytes
    stage_tile_rows<NT>(kp, u, cv.field, b, ext, &tma_bar);
  } else if (!tma) {
    stage_tile4<NT>(kp, u, cv.field, b, ext);
  }
  {
    // the unit rows read every slot of the longest window: the words after
    // each plane's last staged row (up to the next plane) and the pad after
    // the field are zeroed, so that every word a slot can reach is finite
    const int ny_st = ext[1] + kp.yhlo + kp.yhhi;
    const int gap = min(kp.pxy - ny_st * kp.px, kFieldPad);
    const int nplanes = 3 * ext[2];
    for (int k = threadIdx.x; k < nplanes * gap + kFieldPad; k += NT) {
      const int pl = k / max(gap, 1);
      if (k < nplanes * gap) {
        const int cc = pl / ext[2], z = pl - cc * ext[2];
        cv.field[cc * kp.plane + z * kp.pxy + ny_st * kp.px + (k - pl * gap)] = 0.f;
      } else {
        cv.field[3 * kp.plane + (k - nplanes * gap)] = 0.f;
      }
    }
  }
  bool staged = false;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int plane = kp.plane, px = kp.px, pxy = kp.pxy;
  const float bx = kp.beta[0], by = kp.beta[1], bz = kp.beta[2];
  const unsigned fbase = shared_addr(cv.field);
  for (int b0 = e0; b0 < e1; b0 += bs) {
    const int np = min(bs, e1 - b0);
    stage_batch<PB, false, LAP>(cv, b0 == e0 ? rfirst : load_rec(entries, b0, np), np, b0,
                                entries, d0x, nullptr, lapc);
    const int R = build_schedule<PB, NT>(cv, ss, np);  // synchronises
    cp_async_wait_all();                            // field (first batch), x-distances
    // One thread waits (bounded) for the staged field; the block learns the
    // outcome at the barrier and either goes on or returns as a whole.
    int timed_out = 0;
    const bool first_wait = (tma || rows) && !staged;
    if (first_wait && threadIdx.x == 0) {
      bool ok = mbar_wait_ns(&tma_bar, 0, kp.wait_ns);
      if (!ok) {
        mbar_wait_ns(&tma_bar, 0, kp.wait_ns);  // once more for the copy in flight
      } else if (kp.debug_stall) {
        ok = mbar_wait_ns(&stall_bar, 0, kp.wait_ns);  // nothing arrives: runs out
      }
      if (!ok) {
        erpp_set_err(err, ERPP_ERRBIT_TIMEOUT);
        timed_out = 1;
      }
    }
    staged = staged || first_wait;
    if (__syncthreads_or(timed_out)) return (tma || rows) ? 3 : 1;
    // the phase has completed: every thread observes it (acquire of the
    // copied field), which returns at once
    if (first_wait && threadIdx.x != 0) mbar_try_wait(&tma_bar, 0);
    for (int r = 0; r < R; ++r) {
      const uint16_t ui = cv.sched[r * NT + warp * 32 + lane];
      const bool active = ui != kEmpty;
      UnitRows ur = {0, 0, 0, 0, 0.f, 0.f};
      int k = 0, uz = 0;
      float ex[XM], e2[LAP ? XM : 1];
      // LAP: the y-window's mean and variance and the plane's factor
      float my = 0.f, vy = 0.f, pz = 0.f;
#pragma unroll
      for (int q = 0; q < XM; ++q) ex[q] = 0.f;
#pragma unroll
      for (int q = 0; q < (LAP ? XM : 1); ++q) e2[q] = 0.f;
      if (active) {
        const uint32_t w = cv.unit[ui];
        k = (int)(w & 1023u);
        const int z = (int)((w >> 10) & 15u);
        uz = z;
        const Piece4 pc = unpack4(cv.rec[k]);
        const float dx0 = cv.dxb[k];
        make_ex<XM>(pc, dx0, bx, ex);
        ur.base = (pc.z0 + z) * pxy + pc.y0 * px + pc.x0;
        ur.ly = pc.ly;
        ur.lx = pc.lx;
        ur.rot = (int)(w >> 31);
        ur.d0y = pc.d0y;
        const float dz = pc.d0z + (float)z;
        ur.ezz = bz * dz * dz;
        if constexpr (LAP) {
          const float4 c0 = cv.lcb[2 * k], c1 = cv.lcb[2 * k + 1];
#pragma unroll
          for (int q = 0; q < XM; ++q) {
            const float du = dx0 + (float)(pc.qa + q) - c0.x;
            e2[q] = ex[q] * (kp.lap_k[0] * fmaf(du, du, -c0.y));
          }
          my = c0.z;
          vy = c0.w;
          const float dzz = dz - c1.x;
          pz = kp.lap_k[2] * fmaf(dzz, dzz, -c1.y);
        }
      }
      const int rows = __reduce_max_sync(0xffffffffu, (unsigned)ur.ly);
      // Straight-line rows: rows past the unit's own length get weight 0,
      // the rotated walk wraps by a select.  Empty lanes read from column
      // `lane` (their own bucket) and their sums are dropped.  Rows 1.. are
      // summed in row order and the first row's term is added at the end, so
      // that the unit's sum does not depend on where its walk started.
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f;
      float l0 = 0.f, l1 = 0.f, l2 = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f;  // LAP
      const unsigned pl4 = 4u * (unsigned)plane, px4 = 4u * (unsigned)px;
      const unsigned abase = fbase + 4u * (unsigned)(active ? ur.base : lane);
      const unsigned aend = abase + px4 * (unsigned)ur.ly;
      // the rows, visiting the slots of the longest window in the warp
      auto unit_rows = [&](auto nq) {
        constexpr int NQ = decltype(nq)::value;
        unsigned ar = abase + px4 * (unsigned)ur.rot;
        float dy = ur.d0y + (float)ur.rot;
#pragma unroll 1
        for (int t = 0; t < rows; ++t) {
          const float e = exp2f(-fmaf(by * dy, dy, ur.ezz));
          const bool in = t < ur.ly;
          const float wr = in ? e : 0.f;
          float x0 = 0.f, x1 = 0.f, x2 = 0.f;
          float y0 = 0.f, y1 = 0.f, y2 = 0.f;
          if constexpr (LAP)
            row_dot2<0, XM, NQ>(ar, ar + pl4, ar + 2 * pl4, ex, e2, x0, x1, x2, y0, y1, y2);
          else
            row_dot<0, XM, NQ>(ar, ar + pl4, ar + 2 * pl4, ex, x0, x1, x2);
          // LAP: the row's Laplacian term, (P_y + P_z) x_c + y_c
          float pr = 0.f;
          if (LAP) {
            const float ddy = dy - my;
            pr = fmaf(kp.lap_k[1], fmaf(ddy, ddy, -vy), pz);
          }
          if (in && ar == abase) {
            r0 = wr * x0;
            r1 = wr * x1;
            r2 = wr * x2;
            if (LAP) {
              q0 = wr * fmaf(pr, x0, y0);
              q1 = wr * fmaf(pr, x1, y1);
              q2 = wr * fmaf(pr, x2, y2);
            }
          } else {
            a0 = fmaf(wr, x0, a0);
            a1 = fmaf(wr, x1, a1);
            a2 = fmaf(wr, x2, a2);
            if (LAP) {
              l0 = fmaf(wr, fmaf(pr, x0, y0), l0);
              l1 = fmaf(wr, fmaf(pr, x1, y1), l1);
              l2 = fmaf(wr, fmaf(pr, x2, y2), l2);
            }
          }
          ar += px4;
          dy += 1.f;
          const bool wrap = ar == aend;
          ar = wrap ? abase : ar;
          dy = wrap ? ur.d0y : dy;
        }
      };
      if (LMIN < XM && __all_sync(0xffffffffu, ur.lx <= LMIN))
        unit_rows(std::integral_constant<int, LMIN>());
      else
        unit_rows(std::integral_constant<int, XM>());
      if (active) {
        // the unit's own slot (piece k, plane uz): no two units share one
        float* pa = cv.pacc + uz * PB + k;
        pa[0] = a0 + r0;
        pa[tzs * PB] = a1 + r1;
        pa[2 * tzs * PB] = a2 + r2;
        if (LAP) {
          pa[3 * tzs * PB] = l0 + q0;
          pa[4 * tzs * PB] = l1 + q1;
          pa[5 * tzs * PB] = l2 + q2;
        }
      }
    }
    __syncthreads();
    // each piece's sums, its planes added in plane order, at the place of its
    // record (the particle adds its pieces later, in piece order): the result
    // does not depend on the order in which units ran
    for (int k = threadIdx.x; k < np; k += NT) {
      const int lz = unpack4(cv.rec[k]).lz;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int z = 0; z < lz; ++z) {
        s0 += cv.pacc[z * PB + k];
        s1 += cv.pacc[(tzs + z) * PB + k];
        s2 += cv.pacc[(2 * tzs + z) * PB + k];
      }
      up_part[b0 + k] = make_float4(s0, s1, s2, 0.f);
      if (LAP) {
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        for (int z = 0; z < lz; ++z) {
          t0 += cv.pacc[(3 * tzs + z) * PB + k];
          t1 += cv.pacc[(4 * tzs + z) * PB + k];
          t2 += cv.pacc[(5 * tzs + z) * PB + k];
        }
        lap_part[b0 + k] = make_float4(t0, t1, t2, 0.f);
      }
    }
    __syncthreads();
  }
  return (tma || rows) ? 2 : 0;
}

template <int XM, int LMIN, int XW, int NT, bool LAP, int PB>
__global__ void __launch_bounds__(NT, LAP ? 2 : 768 / NT) k_gather4(
    erpp_kparams kp, const float* __restrict__ u, const __grid_constant__ CUtensorMap tmap,
    int use_tma, const int32_t* __restrict__ start, const int4* __restrict__ entries,
    int64_t ecap, const float* __restrict__ d0x, const float4* __restrict__ lapc,
    float4* __restrict__ up_part, float4* __restrict__ lap_part, uint32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SchedState ss;
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ __align__(8) uint64_t stall_bar;  // debug_stall only: never completed
  gather_tile4<XM, LMIN, XW, NT, LAP, PB>(kp, blockIdx.x, u, &tmap, use_tma, start, entries,
                                          ecap, d0x, lapc, up_part, lap_part, err, smem_raw, ss,
                                          tma_bar, stall_bar);
}

// MODE 0: 32-bit fixed point (FP32 atomics on dense tiles); MODE 1: split
// high / low fixed-point words (the compensated mode).
// CL: the launch groups the nt[0] x-tiles of one (y, z) tile row into a
// thread-block cluster (rank = x-tile): once every block of the row has
// formed its final values in shared memory, each block adds its x-neighbours'
// halo columns to its own rim columns straight from their shared memory, in a
// fixed order (own, left, right), so that no x-strip is written and
// k_merge_cols is not needed; the y-halo rows, which then hold the diagonal
// neighbours' corner columns too, still leave as y-strips for k_merge_rows.
// Requires rows of a multiple of 4 nodes and 16-byte aligned S and strips
// (the host launches CL only then).
// Result of accumulating one tile's pieces in shared memory.
struct TileAcc {
  bool any;         // the tile has pieces
  bool fixedp;      // 32-bit fixed point (else FP32 values)
  float inv_scale;  // fixed point: value of one unit of the sums
};

// Accumulates the pieces of `tile` into the staged tile in shared memory
// (cleared first): 32-bit fixed-point integers or FP32 values on dense tiles
// (MODE 0), or high / low fixed-point sums converted to FP32 in place at the
// end (MODE 1).  Called by the whole block.
template <int XM, int LMIN, int XW, int MODE, int NT>
__device__ __forceinline__ TileAcc scatter_tile(const erpp_kparams& kp, int tile,
                                                const Carve<Batch<XW>::kPB>& cv, SchedState& ss,
                                                float* red,
                                                const int32_t* __restrict__ start,
                                                const int4* __restrict__ entries, int64_t ecap,
                                                const float* __restrict__ d0x,
                                                const float4* __restrict__ fscat) {
  constexpr int NW = NT / 32;
  constexpr int PB = Batch<XW>::kPB;
  float* smem = cv.field;
  const int e0 = start[tile];
  const int e1 = (int)min((int64_t)start[tile + 1], ecap);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int plane = kp.plane, px = kp.px, pxy = kp.pxy;
  const bool any = e0 < e1;
  const bool fixedp = (e1 - e0) <= (MODE == 0 ? kDenseTile : kSplitMaxPieces);
  // batches of PB pieces, the remainder last: at about 1.8 units per piece a
  // full batch nearly fills two rounds of 256 lanes, where an even split of
  // a 370-piece tile needs two rounds for each half
  const int bs = any ? PB : 1;
  const int4 rfirst = load_rec(entries, e0, min(bs, e1 - e0));  // overlaps the clearing
  float scale = 1.f, inv_scale = 1.f;
  {
    const int total = (MODE == 1 ? 6 : 3) * plane;
    float4* s4 = reinterpret_cast<float4*>(smem);
    for (int k = threadIdx.x; k < total / 4; k += NT) s4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int wide_sh = 0;  // MODE 1: node sums are in units of 2^-(sh + 31)
  if (any) {
    // Fixed-point scale from the tile's force bound B = sum of max |f| over
    // its pieces (a node receives at most one contribution per piece):
    // B = m 2^ex2 (m in [0.5, 1)) gives factors G below 2^30 (MODE 0: no
    // 32-bit node sum of the products' high words can overflow) or 2^31
    // (MODE 1: no 64-bit node sum of the full products can), whatever the
    // number of pieces.  A tile of one batch sums B from the staged forces, a
    // larger one by a pass over its entries first.
    const bool single = (e1 - e0) <= PB;
    // B is summed exactly, so that it (and the scale) does not depend on the
    // order of the tile's pieces: the block first takes the largest max|f|,
    // then adds every piece's max|f| as a fixed-point integer scaled to it
    // (each below 2^29, summed in 64 bits).
    // get(j) reads the j-th value of this thread, for j < cnt.
    auto set_scale = [&](auto get, int cnt) {
      float m = 0.f;
      for (int j = 0; j < cnt; ++j) m = fmaxf(m, get(j));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) red[warp] = m;
      __syncthreads();
      float mx = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) mx = fmaxf(mx, red[w]);
      __syncthreads();
      int emx = 0;
      frexpf(mx, &emx);
      long long q = 0;
      if (mx > 0.f)
        for (int j = 0; j < cnt; ++j) q += __float2int_rn(ldexpf(get(j), 29 - emx));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (lane == 0) reinterpret_cast<long long*>(red)[warp] = q;
      __syncthreads();
      long long qs = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) qs += reinterpret_cast<long long*>(red)[w];
      const float B = ldexpf(__ll2float_rn(qs), emx - 29);
      if (B > 0.f) {
        int ex2;
        frexpf(B, &ex2);
        const int sh = min((MODE == 1 ? 31 : 30) - ex2, 120);
        scale = ldexpf(1.f, sh);
        // MODE 0: node sums are in units of scale / 2 (the row weight carries
        // 2^31, the high word drops 2^32); MODE 1: in units of 2^-(sh + 31)
        inv_scale = ldexpf(2.f, -sh);
        wide_sh = sh;
      }
    };
    if (fixedp && !single) {
      const int cnt = (e1 - e0 - (int)threadIdx.x + NT - 1) / NT;
      set_scale([&](int j) { return __ldg(&fscat[__ldg(&entries[e0 + threadIdx.x + j * NT].x)]).w; },
                max(cnt, 0));
    }
    const float bx = kp.beta[0], by = kp.beta[1], bz = kp.beta[2];
    const unsigned fbase = shared_addr(smem);
    for (int b0 = e0; b0 < e1; b0 += bs) {
      const int np = min(bs, e1 - b0);
      stage_batch<PB, true>(cv, b0 == e0 ? rfirst : load_rec(entries, b0, np), np, b0, entries,
                            d0x, fscat);
      const int R = build_schedule<PB, NT>(cv, ss, np);  // synchronises
      cp_async_wait_all();
      __syncthreads();
      if (fixedp && single) {
        const int cnt = (np - (int)threadIdx.x + NT - 1) / NT;
        set_scale([&](int j) { return cv.fsb[threadIdx.x + j * NT].w; }, max(cnt, 0));
      }
      for (int r = 0; r < R; ++r) {
        const uint16_t ui = cv.sched[r * NT + warp * 32 + lane];
        const bool active = ui != kEmpty;
        UnitRows ur = {0, 0, 0, 0, 0.f, 0.f};
        float ex[XM];
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        int G0[XM], G1[XM], G2[XM];
#pragma unroll
        for (int q = 0; q < XM; ++q) {
          ex[q] = 0.f;
          G0[q] = G1[q] = G2[q] = 0;
        }
        if (active) {
          const uint32_t w = cv.unit[ui];
          const int k = (int)(w & 1023u);
          const int z = (int)((w >> 10) & 15u);
          const Piece4 pc = unpack4(cv.rec[k]);
          make_ex<XM>(pc, cv.dxb[k], bx, ex);
          ur.base = (pc.z0 + z) * pxy + pc.y0 * px + pc.x0;
          ur.ly = pc.ly;
          ur.lx = pc.lx;
          ur.rot = (int)(w >> 31);
          ur.d0y = pc.d0y;
          const float dz = pc.d0z + (float)z;
          const float wz = exp2f(-bz * dz * dz);
          const float4 fv = cv.fsb[k];
          f0 = fv.x * wz;
          f1 = fv.y * wz;
          f2 = fv.z * wz;
          if (fixedp) {
#pragma unroll
            for (int q = 0; q < XM; ++q) {
              G0[q] = __float2int_rn(f0 * scale * ex[q]);
              G1[q] = __float2int_rn(f1 * scale * ex[q]);
              G2[q] = __float2int_rn(f2 * scale * ex[q]);
            }
          }
        }
        const int rows = __reduce_max_sync(0xffffffffu, (unsigned)ur.ly);
        // Rows as in the gather: straight line, weight 0 past the unit's
        // length, rotated walk wrapping by a select; empty lanes add zeros at
        // column `lane` (their own bucket).  Slots past the window are skipped.
        const unsigned pl4 = 4u * (unsigned)plane, px4 = 4u * (unsigned)px;
        const unsigned abase = fbase + 4u * (unsigned)(active ? ur.base : lane);
        const unsigned aend = abase + px4 * (unsigned)ur.ly;
        // the rows, visiting the slots of the longest window in the warp
        auto unit_rows = [&](auto nq) {
          constexpr int NQ = decltype(nq)::value;
          unsigned ar = abase + px4 * (unsigned)ur.rot;
          float dy = ur.d0y + (float)ur.rot;
          if (MODE == 1 && fixedp) {
            const unsigned lo = 3u * pl4;  // the low sums follow the three components
#pragma unroll 1
            for (int t = 0; t < rows; ++t) {
              const float e = exp2f(-by * dy * dy);
              const int W = t < ur.ly ? __float2int_rn(e * 2147483648.f) : 0;
              row_red_split<0, XM, LMIN, NQ>(ar, ar + pl4, ar + 2 * pl4, lo, G0, G1, G2, W, ur.lx);
              ar += px4;
              dy += 1.f;
              const bool wrap = ar == aend;
              ar = wrap ? abase : ar;
              dy = wrap ? ur.d0y : dy;
            }
          } else if (fixedp) {
#pragma unroll 1
            for (int t = 0; t < rows; ++t) {
              const float e = exp2f(-by * dy * dy);
              const int W = t < ur.ly ? __float2int_rn(e * 2147483648.f) : 0;
              row_red_fixed<0, XM, LMIN, NQ>(ar, ar + pl4, ar + 2 * pl4, G0, G1, G2, W, ur.lx);
              ar += px4;
              dy += 1.f;
              const bool wrap = ar == aend;
              ar = wrap ? abase : ar;
              dy = wrap ? ur.d0y : dy;
            }
          } else {
#pragma unroll 1
            for (int t = 0; t < rows; ++t) {
              const float e = exp2f(-by * dy * dy);
              const float wy = t < ur.ly ? e : 0.f;
              row_red_f32<0, XM, LMIN, NQ>(ar, ar + pl4, ar + 2 * pl4, ex, f0, f1, f2, wy, ur.lx);
              ar += px4;
              dy += 1.f;
              const bool wrap = ar == aend;
              ar = wrap ? abase : ar;
              dy = wrap ? ur.d0y : dy;
            }
          }
        };
        if (LMIN < XM && __all_sync(0xffffffffu, ur.lx <= LMIN))
          unit_rows(std::integral_constant<int, LMIN>());
        else
          unit_rows(std::integral_constant<int, XM>());
      }
      __syncthreads();
    }
    if (MODE == 1 && fixedp) {
      // high and low sums to FP32 values in place: the node sum is
      // (2^32 H + 2^17 L) 2^-(sh + 31)
      int* hi = reinterpret_cast<int*>(smem);
      const int* lo = hi + 3 * plane;
      const float s_hi = ldexpf(1.f, 1 - wide_sh), s_lo = ldexpf(1.f, -14 - wide_sh);
      for (int k = threadIdx.x; k < 3 * plane; k += NT)
        smem[k] = fmaf((float)hi[k], s_hi, (float)lo[k] * s_lo);
      __syncthreads();
    }
  }
  return TileAcc{any, fixedp, inv_scale};
}

// The scatter of one tile with its write-out, called by the whole block (the
// body of k_scatter4 and of the multi-box scatter).
template <int XM, int LMIN, int XW, int MODE, int NT, bool CL>
__device__ __forceinline__ void scatter_tile4(const erpp_kparams& kp, int tile,
                                              float* __restrict__ S, float* __restrict__ halo,
                                              const int32_t* __restrict__ start,
                                              const int4* __restrict__ entries, int64_t ecap,
                                              const float* __restrict__ d0x,
                                              const float4* __restrict__ fscat,
                                              unsigned char* smem_raw, SchedState& ss,
                                              float* red) {
  constexpr int NW = NT / 32;
  constexpr int PB = Batch<XW>::kPB;
  static_assert(PB <= NT, "a batch holds at most one piece per thread");
  const Carve<PB> cv = carve<PB>(smem_raw, kp.plane, kp.T[2], MODE == 1 ? 6 : 3, false);
  float* smem = cv.field;
  const TileAcc ta =
      scatter_tile<XM, LMIN, XW, MODE, NT>(kp, tile, cv, ss, red, start, entries, ecap, d0x,
                                           fscat);
  const bool any = ta.any, fixedp = ta.fixedp;
  const float inv_scale = ta.inv_scale;
  int b[3], ext[3], tt[3];
  tile_origin4(kp, tile, b, ext, tt);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int plane = kp.plane, px = kp.px, pxy = kp.pxy;
  int* acc_i = reinterpret_cast<int*>(smem);
  // interior once (zeros for empty tiles); halo strips to the buffer:
  // x-strips [3][T_z][T_y + hy][hx] (all staged rows), y-strips [3][T_z][hy][W]
  // (16-byte aligned).
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const int hx = kp.xhlo + kp.xhhi, hy = kp.yhlo + kp.yhhi;
  const int ny_st = ext[1] + hy;
  float* hxs = halo + (size_t)tile * kp.halo_per_tile;
  float* hys = hxs + kp.ystrip_off;
  const bool vec = CL || ((kp.n[0] & 3) == 0 && (ext[0] & 3) == 0 && (b[0] & 3) == 0 &&
                           (kp.T[0] & 3) == 0 && (((uintptr_t)S) & 15) == 0 &&
                           (((uintptr_t)halo) & 15) == 0);
  if (CL || (vec && hx <= 16)) {
    // Aligned rows: the final values are formed in place, then every staged
    // row's interior columns leave by one bulk asynchronous copy (to S, or to
    // the y-strip on a y-halo row) and the hx halo columns of all rows by
    // plain stores (to the x-strip, contiguous per component and plane).
    float4* s4 = reinterpret_cast<float4*>(smem);
    if (any && MODE == 0 && fixedp) {
      const int total4 = 3 * plane / 4;
      for (int k = threadIdx.x; k < total4; k += NT) {
        const int4 q = reinterpret_cast<const int4*>(smem)[k];
        s4[k] = make_float4((float)q.x * inv_scale, (float)q.y * inv_scale,
                            (float)q.z * inv_scale, (float)q.w * inv_scale);
      }
    }
    const unsigned fbase = shared_addr(smem);
    if (CL) {
      // every block of the row has its final values in place
      cluster_arrive();
      cluster_wait();
      const int ntx = kp.nt[0];
      const unsigned rank = cluster_ctarank();
      const unsigned rl = rank == 0 ? ntx - 1 : rank - 1;
      const unsigned rr = rank + 1 == (unsigned)ntx ? 0 : rank + 1;
      const int extl = min((int)(rl + 1) * kp.T[0], kp.n[0]) - (int)rl * kp.T[0];
      const unsigned lbase = mapa_shared(fbase, rl), rbase = mapa_shared(fbase, rr);
      // rim columns: x < xhhi take the left tile's right halo (its column
      // xoff + extl + x), x >= ext - xhlo the right tile's left halo (its
      // column xoff + x - ext); a tile narrower than hx takes both
      const bool allcols = ext[0] < hx;
      const int ncol = allcols ? ext[0] : hx;
      const int njob = 3 * ext[2] * ny_st * ncol;
      for (int j = threadIdx.x; j < njob; j += NT) {
        const int r = j / ncol;
        const int q = j - r * ncol;
        const int x = allcols || q < kp.xhhi ? q : ext[0] - hx + q;
        const int cz = r / ny_st;
        const int y = r - cz * ny_st;
        const int cc = cz / ext[2];
        const int z = cz - cc * ext[2];
        const int row = cc * plane + z * pxy + y * px + kp.xoff;
        float v = smem[row + x];
        if (x < kp.xhhi) v += ld_cluster_f32(lbase + 4u * (unsigned)(row + extl + x));
        if (x >= ext[0] - kp.xhlo) v += ld_cluster_f32(rbase + 4u * (unsigned)(row + x - ext[0]));
        smem[row + x] = v;
      }
      // this block has read its neighbours' halos (they may leave once every
      // block has arrived here)
      cluster_arrive();
    }
    fence_proxy_async_shared();
    __syncthreads();
    const int nrow = 3 * ext[2] * ny_st;
    bool issued = false;
    for (int r = threadIdx.x; r < nrow; r += NT) {
      const int cz = r / ny_st;
      const int y = r - cz * ny_st;
      const int cc = cz / ext[2];
      const int z = cz - cc * ext[2];
      const int so = cc * plane + z * pxy + y * px + kp.xoff;
      const bool yint = y >= kp.yhlo && y < kp.yhlo + ext[1];
      const int yh = y < kp.yhlo ? y : y - ext[1];
      float* drow = yint ? S + cc * nn +
                               ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y - kp.yhlo)) * kp.n[0] +
                               b[0]
                         : hys + (((size_t)cc * kp.T[2] + z) * hy + yh) * kp.T[0];
      bulk_store_s2g(drow, fbase + 4u * (unsigned)so, 4u * (unsigned)ext[0]);
      issued = true;
    }
    if (issued) bulk_commit_wait_read();
    if (CL) {
      // the neighbours have read this block's halo columns
      cluster_wait();
      return;
    }
    if (kp.xclip) return;  // no contributions to the x-halo columns
    const int rpw = 32 / hx;  // staged rows per warp pass
    const int rsub = lane / hx, h = lane - rsub * hx;
    const int col = h < kp.xhlo ? kp.xoff - kp.xhlo + h : kp.xoff + ext[0] + (h - kp.xhlo);
    if (rsub < rpw) {
      for (int cc = 0; cc < 3; ++cc) {
        for (int z = 0; z < ext[2]; ++z) {
          const float* srow = smem + cc * plane + z * pxy + col;
          float* xs = hxs + ((size_t)cc * kp.T[2] + z) * (kp.T[1] + hy) * hx + h;
          for (int y = warp * rpw + rsub; y < ny_st; y += NW * rpw) xs[y * hx] = srow[y * px];
        }
      }
    }
    return;
  }
  // General rows: per staged row the lanes take jobs: 16-byte chunks of the
  // interior columns (to S, or to the y-strip on a y-halo row) when
  // everything is aligned, else single words; then the hx halo columns (to
  // the x-strip).
  const int nvec = vec ? ext[0] >> 2 : 0;
  const int jobs = nvec + (vec ? 0 : ext[0]) + (kp.xclip ? 0 : hx);
  auto value = [&](int idx) -> float {
    if (!any) return 0.f;
    if (MODE == 0 && fixedp) return (float)acc_i[idx] * inv_scale;
    return smem[idx];
  };
  for (int cc = 0; cc < 3; ++cc) {
    for (int z = 0; z < ext[2]; ++z) {
      for (int y = warp; y < ny_st; y += NW) {
        const int so = cc * plane + z * pxy + y * px;  // staged row start
        const bool yint = y >= kp.yhlo && y < kp.yhlo + ext[1];
        const int yh = y < kp.yhlo ? y : y - ext[1];  // y-strip row when !yint
        float* drow = yint ? S + cc * nn +
                                 ((size_t)(b[2] + z) * kp.n[1] + (b[1] + y - kp.yhlo)) * kp.n[0] +
                                 b[0]
                           : hys + (((size_t)cc * kp.T[2] + z) * hy + yh) * kp.T[0];
        float* xrow = hxs + (((size_t)cc * kp.T[2] + z) * (kp.T[1] + hy) + y) * hx;
        for (int j = lane; j < jobs; j += 32) {
          if (j < nvec) {
            const int i0 = so + kp.xoff + 4 * j;
            float4 v;
            if (!any) {
              v = make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (MODE == 0 && fixedp) {
              const int4 q = *reinterpret_cast<const int4*>(acc_i + i0);
              v = make_float4((float)q.x * inv_scale, (float)q.y * inv_scale,
                              (float)q.z * inv_scale, (float)q.w * inv_scale);
            } else {
              v = *reinterpret_cast<const float4*>(smem + i0);
            }
            *reinterpret_cast<float4*>(drow + 4 * j) = v;
          } else {
            const int sj = j - nvec;
            if (!vec && sj < ext[0]) {
              drow[sj] = value(so + kp.xoff + sj);
            } else {
              const int h = vec ? sj : sj - ext[0];
              const int col = h < kp.xhlo ? kp.xoff - kp.xhlo + h : kp.xoff + ext[0] + (h - kp.xhlo);
              xrow[h] = value(so + col);
            }
          }
        }
      }
    }
  }
}

template <int XM, int LMIN, int XW, int MODE, int NT, bool CL>
__global__ void __launch_bounds__(NT, MODE == 0 ? 1024 / NT : 2) k_scatter4(
    erpp_kparams kp, float* __restrict__ S, float* __restrict__ halo,
    const int32_t* __restrict__ start, const int4* __restrict__ entries, int64_t ecap,
    const float* __restrict__ d0x, const float4* __restrict__ fscat) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SchedState ss;
  __shared__ __align__(8) float red[2 * (NT / 32)];  // per-warp partials (8-byte ones too)
  scatter_tile4<XM, LMIN, XW, MODE, NT, CL>(kp, blockIdx.x, S, halo, start, entries, ecap, d0x,
                                            fscat, smem_raw, ss, red);
}

// Adds the scatter's halo strips onto the tiles they belong to, in two
// phases (stream order, each node updated by one thread per phase, so the
// result is deterministic), one block per tile, periodic in x and y:
//   k_merge_rows: rows within yhhi / yhlo of the tile's lower / upper edge
//     receive the y-strips of the lower / upper neighbour (whole rows, 16-byte
//     chunks when aligned);
//   k_merge_cols: columns within xhhi / xhlo of the left / right edge receive
//     the x-strips of the left / right neighbour (same rows) and, in the rim
//     rows, the x-strips of the diagonal neighbours (their y-halo rows).
// A thread keeps one (row, chunk) or (row, column) job for every component
// and plane of the tile, so the index arithmetic is done once per job.
__device__ __forceinline__ int tile_id(const erpp_kparams& kp, int tx, int ty, int tz) {
  return (tz * kp.nt[1] + ty) * kp.nt[0] + tx;
}

constexpr int kMergeThreads = 128;

__device__ __forceinline__ void merge_rows_tile(const erpp_kparams& kp, int tile,
                                                float* __restrict__ S,
                                                const float* __restrict__ halo) {
  int b[3], ext[3], t[3];
  tile_origin4(kp, tile, b, ext, t);
  const int W = kp.T[0], hy = kp.yhlo + kp.yhhi;
  const int tyl = t[1] == 0 ? kp.nt[1] - 1 : t[1] - 1;
  const int tyr = t[1] == kp.nt[1] - 1 ? 0 : t[1] + 1;
  const float* hB = halo + (size_t)tile_id(kp, t[0], tyl, t[2]) * kp.halo_per_tile + kp.ystrip_off;
  const float* hT = halo + (size_t)tile_id(kp, t[0], tyr, t[2]) * kp.halo_per_tile + kp.ystrip_off;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const size_t nxy = (size_t)kp.n[0] * kp.n[1];
  const int ycut = ext[1] - kp.yhlo;
  // rim rows: [0, min(yhhi, ext)) and [max(ycut, yhhi), ext) (all rows when ext < hy)
  const int na = min(kp.yhhi, ext[1]);
  const int nb = ext[1] - max(ycut, na);
  const bool vec = (W & 3) == 0 && (ext[0] & 3) == 0 && (kp.n[0] & 3) == 0 && (b[0] & 3) == 0 &&
                   (((uintptr_t)S) & 15) == 0 && (((uintptr_t)halo) & 15) == 0;
  const int per_row = vec ? ext[0] >> 2 : ext[0];
  const int njobs = (na + nb) * per_row;
  const size_t qstride = (size_t)hy * W;  // one component-plane of the y-strips
  for (int i = threadIdx.x; i < njobs; i += kMergeThreads) {
    const int r = i / per_row;
    const int j = i - r * per_row;
    const int y = r < na ? r : max(ycut, na) + (r - na);
    const bool yl = y < kp.yhhi, yr = y >= ycut;
    float* drow = S + (size_t)b[2] * nxy + (size_t)(b[1] + y) * kp.n[0] + b[0];
    const float* brow = hB + (size_t)(kp.yhlo + y) * W;
    const float* trow = hT + (size_t)(y - ycut) * W;
    for (int cc = 0; cc < 3; ++cc) {
      for (int z = 0; z < ext[2]; ++z) {
        float* d = drow + cc * nn + z * nxy;
        const size_t q = (size_t)(cc * kp.T[2] + z) * qstride;
        if (vec) {
          float4 v = reinterpret_cast<float4*>(d)[j];
          if (yl) {
            const float4 a = reinterpret_cast<const float4*>(brow + q)[j];
            v.x += a.x; v.y += a.y; v.z += a.z; v.w += a.w;
          }
          if (yr) {
            const float4 a = reinterpret_cast<const float4*>(trow + q)[j];
            v.x += a.x; v.y += a.y; v.z += a.z; v.w += a.w;
          }
          reinterpret_cast<float4*>(d)[j] = v;
        } else {
          float v = d[j];
          if (yl) v += brow[q + j];
          if (yr) v += trow[q + j];
          d[j] = v;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_rows(erpp_kparams kp, float* __restrict__ S,
                                                              const float* __restrict__ halo) {
  merge_rows_tile(kp, blockIdx.x, S, halo);
}

__device__ __forceinline__ void merge_cols_tile(const erpp_kparams& kp, int tile,
                                                float* __restrict__ S,
                                                const float* __restrict__ halo) {
  int b[3], ext[3], t[3];
  tile_origin4(kp, tile, b, ext, t);
  const int hx = kp.xhlo + kp.xhhi, hy = kp.yhlo + kp.yhhi;
  const int Ty = kp.T[1];
  const int txl = t[0] == 0 ? kp.nt[0] - 1 : t[0] - 1;
  const int txr = t[0] == kp.nt[0] - 1 ? 0 : t[0] + 1;
  const int tyl = t[1] == 0 ? kp.nt[1] - 1 : t[1] - 1;
  const int tyr = t[1] == kp.nt[1] - 1 ? 0 : t[1] + 1;
  auto strip = [&](int tx, int ty) {
    return halo + (size_t)tile_id(kp, tx, ty, t[2]) * kp.halo_per_tile;
  };
  const int exty_l = min((tyl + 1) * Ty, kp.n[1]) - tyl * Ty;
  const int xcut = ext[0] - kp.xhlo, ycut = ext[1] - kp.yhlo;
  const size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  const size_t nxy = (size_t)kp.n[0] * kp.n[1];
  const bool allcols = ext[0] < hx;
  const int ncol = allcols ? ext[0] : hx;
  const size_t qstride = (size_t)(Ty + hy) * hx;  // one component-plane of the x-strips
  for (int i = threadIdx.x; i < ext[1] * ncol; i += kMergeThreads) {
    const int y = i / ncol;
    const int j = i - y * ncol;
    const int x = allcols || j < kp.xhhi ? j : xcut + (j - kp.xhhi);
    const bool xl = x < kp.xhhi, xr = x >= xcut;
    if (!(xl || xr)) continue;
    const bool yl = y < kp.yhhi, yr = y >= ycut;
    // offsets of this node's entries in the six strips (same for every plane)
    const int cl = kp.xhlo + x, cr = x - xcut;
    const float* pL = strip(txl, t[1]) + (y + kp.yhlo) * hx + cl;
    const float* pR = strip(txr, t[1]) + (y + kp.yhlo) * hx + cr;
    const float* pLB = strip(txl, tyl) + (exty_l + kp.yhlo + y) * hx + cl;
    const float* pRB = strip(txr, tyl) + (exty_l + kp.yhlo + y) * hx + cr;
    const float* pLT = strip(txl, tyr) + (y - ycut) * hx + cl;
    const float* pRT = strip(txr, tyr) + (y - ycut) * hx + cr;
    float* drow = S + (size_t)b[2] * nxy + (size_t)(b[1] + y) * kp.n[0] + b[0] + x;
    for (int cc = 0; cc < 3; ++cc) {
      for (int z = 0; z < ext[2]; ++z) {
        const size_t q = (size_t)(cc * kp.T[2] + z) * qstride;
        float add = 0.f;
        if (xl) add += pL[q];
        if (xr) add += pR[q];
        if (xl && yl) add += pLB[q];
        if (xr && yl) add += pRB[q];
        if (xl && yr) add += pLT[q];
        if (xr && yr) add += pRT[q];
        float* d = drow + cc * nn + z * nxy;
        *d += add;
      }
    }
  }
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_cols(erpp_kparams kp, float* __restrict__ S,
                                                              const float* __restrict__ halo) {
  merge_cols_tile(kp, blockIdx.x, S, halo);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of the field u for the staged box [PX x NY x T_z x 3] (the
// shared layout without plane padding).  False when the layout or the
// alignment does not allow it (the kernels then stage with cp.async).
bool field_tensor_map(const erpp_kparams& kp, const float* u, CUtensorMap* map) {
  const int ny_st = kp.T[1] + kp.yhlo + kp.yhhi;
  if ((kp.n[0] & 3) || (kp.T[0] & 3) || (kp.xoff & 3) || kp.pxy != kp.px * ny_st ||
      (((uintptr_t)u) & 15) || kp.px > 256 || ny_st > 256 || kp.T[2] > 256)
    return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)kp.n[0], (cuuint64_t)kp.n[1], (cuuint64_t)kp.n[2], 3};
  const cuuint64_t strides[3] = {(cuuint64_t)kp.n[0] * 4, (cuuint64_t)kp.n[0] * kp.n[1] * 4,
                                 (cuuint64_t)kp.n[0] * kp.n[1] * kp.n[2] * 4};
  const cuuint32_t box[4] = {(cuuint32_t)kp.px, (cuuint32_t)ny_st, (cuuint32_t)kp.T[2], 3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(u), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int XM, int LMIN, int XW, int NT, bool LAP, int PB>
cudaError_t gather4_nt(erpp_ctx* ctx, const float* u, cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  if (LAP && (!ctx->lapc || !ctx->lap_part)) return cudaErrorInvalidValue;
  const size_t sm = carve_bytes<PB>(kp.plane, kp.T[2], 3, true, LAP);
  auto kern = k_gather4<XM, LMIN, XW, NT, LAP, PB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const int use_tma = field_tensor_map(kp, u, &map) ? 1 : 0;
  ++ctx->launches;
  kern<<<kp.ntiles, NT, sm, st>>>(kp, u, map, use_tma, ctx->tile_start, ctx->entries,
                                  ctx->entries_cap, ctx->d0x, ctx->lapc, ctx->up_part,
                                  ctx->lap_part, ctx->err);
  return cudaGetLastError();
}

// Blocks of the gather per SM for a dynamic shared-memory size (the SM's
// 228 KB, 1 KB reserved and about 0.4 KB of static shared memory per block).
inline int gather_blocks_per_sm(size_t smem) {
  return (int)((228u * 1024u) / (smem + 1024u + 512u));
}
// The gather takes batches of twice the pieces when that costs no block per
// SM (at most three: its registers allow three 256-thread blocks): more units
// per batch fill the schedule's rounds better.
inline bool gather_big_batch(size_t small, size_t big) {
  return std::min(gather_blocks_per_sm(big), 3) >= std::min(gather_blocks_per_sm(small), 3);
}

// LAP (the general force's gather) always runs 256-thread blocks.
template <int XM, int LMIN, int XW, bool LAP = false>
cudaError_t gather4(erpp_ctx* ctx, const float* u, cudaStream_t st) {
  constexpr int PB = Batch<XW>::kPB;
  if constexpr (LAP) {
    return gather4_nt<XM, LMIN, XW, 256, true, PB>(ctx, u, st);
  } else {
    if (ctx->kp.nthreads == 512) return gather4_nt<XM, LMIN, XW, 512, false, PB>(ctx, u, st);
    const erpp_kparams& kp = ctx->kp;
    if (gather_big_batch(carve_bytes<PB>(kp.plane, kp.T[2], 3, true),
                         carve_bytes<2 * PB>(kp.plane, kp.T[2], 3, true)))
      return gather4_nt<XM, LMIN, XW, 256, false, 2 * PB>(ctx, u, st);
    return gather4_nt<XM, LMIN, XW, 256, false, PB>(ctx, u, st);
  }
}

// Launches k_scatter4; CL: as thread-block clusters of the nt[0] x-tiles of a
// tile row (returns cudaErrorNotSupported, launching nothing, when such
// clusters cannot be resident).
template <int XM, int LMIN, int XW, int MODE, int NT, bool CL>
cudaError_t scatter4_mode(erpp_ctx* ctx, float* S, cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  const size_t sm = carve_bytes<Batch<XW>::kPB>(kp.plane, kp.T[2], MODE == 1 ? 6 : 3, false);
  auto kern = k_scatter4<XM, LMIN, XW, MODE, NT, CL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (!CL) {
    ++ctx->launches;
    kern<<<kp.ntiles, NT, sm, st>>>(kp, S, ctx->halo, ctx->tile_start, ctx->entries,
                                    ctx->entries_cap, ctx->d0x, ctx->fscat);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)kp.ntiles);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)kp.nt[0];
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (ctx->cluster_probe == 0) {
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) cudaGetLastError();
    ctx->cluster_probe = (e == cudaSuccess && nclusters >= 1) ? 1 : 2;
  }
  if (ctx->cluster_probe != 1) return cudaErrorNotSupported;
  ++ctx->launches;
  return cudaLaunchKernelEx(&cfg, kern, kp, S, ctx->halo, (const int32_t*)ctx->tile_start,
                            (const int4*)ctx->entries, ctx->entries_cap,
                            (const float*)ctx->d0x, (const float4*)ctx->fscat);
}

template <int XM, int LMIN, int XW, bool CL>
cudaError_t scatter4(erpp_ctx* ctx, float* S, cudaStream_t st) {
  const bool big = ctx->kp.nthreads == 512;
  if (ctx->kp.kahan)
    return big ? scatter4_mode<XM, LMIN, XW, 1, 512, CL>(ctx, S, st)
               : scatter4_mode<XM, LMIN, XW, 1, 256, CL>(ctx, S, st);
  return big ? scatter4_mode<XM, LMIN, XW, 0, 512, CL>(ctx, S, st)
             : scatter4_mode<XM, LMIN, XW, 0, 256, CL>(ctx, S, st);
}

template <bool CL>
cudaError_t scatter4_variant(erpp_ctx* ctx, float* S, cudaStream_t st, int variant) {
  switch (variant) {
    case 0: return scatter4<7, 6, 8, CL>(ctx, S, st);
    case 1: return scatter4<7, 5, 8, CL>(ctx, S, st);
    case 2: return scatter4<10, 9, 16, CL>(ctx, S, st);
    case 3: return scatter4<10, 8, 16, CL>(ctx, S, st);
    default: break;
  }
  if constexpr (!CL) {  // windows cut at x-tile boundaries (never clustered)
    if (variant == 5) return scatter4<7, 1, 8, CL>(ctx, S, st);
    if (variant == 6) return scatter4<10, 1, 16, CL>(ctx, S, st);
  }
  return scatter4<16, 1, 16, CL>(ctx, S, st);
}

// The x-halo exchange through clusters needs whole 16-byte rows (every
// tile's start and width a multiple of 4 nodes), aligned source and strips,
// and a row of at most 8 x-tiles (the portable cluster size).
bool cluster_eligible(const erpp_ctx* ctx, const float* S) {
  const erpp_kparams& kp = ctx->kp;
  return ctx->scatter_mode == ERPP_SCATTER_CLUSTER && !kp.xclip && kp.nt[0] >= 1 &&
         kp.nt[0] <= 8 &&
         (kp.n[0] & 3) == 0 && (kp.T[0] & 3) == 0 && (((uintptr_t)S) & 15) == 0 &&
         (((uintptr_t)ctx->halo) & 15) == 0;
}

// ---- Many boxes in one launch (batched boxes) ----
// One box of a multi-box launch, in device memory: its kernel parameters,
// the field's tensor map and its buffers (those of its context).
struct __align__(64) BoxTiles {
  CUtensorMap tmap;
  erpp_kparams kp;
  const float* u;
  float* S;
  float* halo;
  const int32_t* start;
  const int4* entries;
  int64_t ecap;
  const float* d0x;
  const float4* fscat;
  float4* up_part;
  uint32_t* err;
  int use_tma;
};

// Persistent blocks pull (box, tile) work items from a counter that only
// grows, so every block ends once the items are used up: no block waits on
// another.  The items are ordered by cost (denser boxes first); each is the
// single-box tile body with the box's parameters and buffers.
template <int XM, int LMIN, int XW>
__global__ void __launch_bounds__(256, 3) k_gather4_multi(const BoxTiles* __restrict__ boxes,
                                                          const int2* __restrict__ items,
                                                          int nitems, int* __restrict__ counter) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SchedState ss;
  __shared__ __align__(8) uint64_t tma_bar;
  __shared__ __align__(8) uint64_t stall_bar;
  __shared__ int item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = item;
    if (it >= nitems) break;
    const int2 bt = items[it];
    const BoxTiles& B = boxes[bt.x];
    const int r = gather_tile4<XM, LMIN, XW, 256, false, Batch<XW>::kPB>(
        B.kp, bt.y, B.u, &B.tmap, B.use_tma, B.start, B.entries, B.ecap, B.d0x, nullptr,
        B.up_part, nullptr, B.err, smem_raw, ss, tma_bar, stall_bar);
    // every thread is done with the tile, its barriers and `item`
    __syncthreads();
    if (r & 1) break;  // a bounded wait ran out (recorded): the block stops
    if (threadIdx.x == 0 && (r & 2)) {
      mbar_inval(&tma_bar);
      if (B.kp.debug_stall) mbar_inval(&stall_bar);
    }
  }
}

template <int XM, int LMIN, int XW>
__global__ void __launch_bounds__(256, 4) k_scatter4_multi(const BoxTiles* __restrict__ boxes,
                                                           const int2* __restrict__ items,
                                                           int nitems, int* __restrict__ counter) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ SchedState ss;
  __shared__ __align__(8) float red[2 * (256 / 32)];
  __shared__ int item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = item;
    if (it >= nitems) break;
    const int2 bt = items[it];
    const BoxTiles& B = boxes[bt.x];
    scatter_tile4<XM, LMIN, XW, 0, 256, false>(B.kp, bt.y, B.S, B.halo, B.start, B.entries,
                                               B.ecap, B.d0x, B.fscat, smem_raw, ss, red);
    // every thread is done with the tile's shared memory and `item`
    __syncthreads();
  }
}

// The halo merges of every box's tiles: one block per (box, tile) item
// (x-windows cut at x-tile boundaries leave no x-strips to merge).
__global__ void __launch_bounds__(kMergeThreads) k_merge_rows_multi(
    const BoxTiles* __restrict__ boxes, const int2* __restrict__ items) {
  const int2 bt = items[blockIdx.x];
  const BoxTiles& B = boxes[bt.x];
  merge_rows_tile(B.kp, bt.y, B.S, B.halo);
}
__global__ void __launch_bounds__(kMergeThreads) k_merge_cols_multi(
    const BoxTiles* __restrict__ boxes, const int2* __restrict__ items) {
  const int2 bt = items[blockIdx.x];
  const BoxTiles& B = boxes[bt.x];
  if (!B.kp.xclip) merge_cols_tile(B.kp, bt.y, B.S, B.halo);
}

}  // namespace

namespace erpp {

// Window-length variants of the unit-schedule kernels: x-windows of 6-7 nodes
// (cutoff 3 sigma_R at sigma_R = dx; 5-7 when rounding leaves c' just below 3)
// and 9-10 nodes (sigma_R = 1.5 dx), else a generic form testing every slot.
int variant4(const erpp_kparams& kp) {
  // windows cut at x-tile boundaries can be shorter than any window: every
  // slot is tested
  if (kp.xclip) return kp.xxs <= 7 ? 5 : (kp.xxs <= 10 ? 6 : 4);
  if (kp.xxs <= 7 && kp.xlmin >= 6) return 0;
  if (kp.xxs <= 7 && kp.xlmin >= 5) return 1;
  if (kp.xxs <= 10 && kp.xlmin >= 9) return 2;
  if (kp.xxs <= 10 && kp.xlmin >= 8) return 3;
  return 4;
}

// Batch width of the design-4 kernels: 8 for the variants of windows of at
// most 7 nodes (0, 1, 5), else 16.
int xw4(const erpp_kparams& kp) {
  const int v = variant4(kp);
  return (v == 0 || v == 1 || v == 5) ? 8 : 16;
}

// Dynamic shared memory of the design-4 kernels (host side of the carve),
// for the batch width the launched variant uses; a general-force context's
// gather also stages the Laplacian moments and sums.
size_t smem_bytes4(const erpp_kparams& kp, int copies, bool gather) {
  const bool lap = gather && kp.full_force;
  const int tz = kp.plane / kp.pxy;
  if (gather)  // the smaller batch: the launch takes the larger only when it fits as well
    return xw4(kp) == 8 ? carve_bytes<Batch<8>::kPB>(kp.plane, tz, copies, true, lap)
                        : carve_bytes<Batch<16>::kPB>(kp.plane, tz, copies, true, lap);
  return xw4(kp) == 8 ? carve_bytes<Batch<8>::kPB>(kp.plane, tz, copies, false, lap)
                      : carve_bytes<Batch<16>::kPB>(kp.plane, tz, copies, false, lap);
}

template <bool LAP>
cudaError_t gather4_variant(erpp_ctx* ctx, const float* u, cudaStream_t st) {
  switch (variant4(ctx->kp)) {
    case 0: return gather4<7, 6, 8, LAP>(ctx, u, st);
    case 1: return gather4<7, 5, 8, LAP>(ctx, u, st);
    case 2: return gather4<10, 9, 16, LAP>(ctx, u, st);
    case 3: return gather4<10, 8, 16, LAP>(ctx, u, st);
    case 5: return gather4<7, 1, 8, LAP>(ctx, u, st);
    case 6: return gather4<10, 1, 16, LAP>(ctx, u, st);
    default: return gather4<16, 1, 16, LAP>(ctx, u, st);
  }
}

cudaError_t launch_gather_f32_4(erpp_ctx* ctx, const float* u, cudaStream_t st) {
  return gather4_variant<false>(ctx, u, st);
}

cudaError_t launch_gather_lap_f32_4(erpp_ctx* ctx, const float* u, cudaStream_t st) {
  return gather4_variant<true>(ctx, u, st);
}

cudaError_t launch_scatter_f32_4(erpp_ctx* ctx, float* S, cudaStream_t st) {
  const int v = variant4(ctx->kp);
  bool clustered = false;
  cudaError_t e = cudaErrorNotSupported;
  if (cluster_eligible(ctx, S)) {
    e = scatter4_variant<true>(ctx, S, st, v);
    clustered = e == cudaSuccess;
  }
  if (e == cudaErrorNotSupported) e = scatter4_variant<false>(ctx, S, st, v);
  if (e != cudaSuccess) return e;
  ++ctx->launches;
  k_merge_rows<<<ctx->kp.ntiles, kMergeThreads, 0, st>>>(ctx->kp, S, ctx->halo);
  if (!clustered && !ctx->kp.xclip) {
    ++ctx->launches;
    k_merge_cols<<<ctx->kp.ntiles, kMergeThreads, 0, st>>>(ctx->kp, S, ctx->halo);
  }
  return cudaGetLastError();
}


// ---- multi-box launches ----
struct Multi4 {
  BoxTiles* boxes = nullptr;      // device: tile kernels' view of every box
  erpp_box_dev* pboxes = nullptr; // device: particle kernels' view
  int2* items = nullptr;          // device: (box, tile), densest boxes first
  int2* pitems = nullptr;         // device: (box, first particle), 256 each
  int* counter = nullptr;         // device: [gather, scatter]
  int nbox = 0;
  int nitems = 0;
  int npitems = 0;
  int variant = 0;
  size_t smem_g = 0, smem_s = 0;
  int grid_g = 0, grid_s = 0;
};

// The window variant one launch can serve for every box: the boxes' own
// variants must share the longest window (0, 1: 7 nodes; 2, 3: 10 nodes); of
// two, the one that tests more slots (1, 3) serves both.  -1: none.
int multi4_variant(erpp_ctx* const* ctx, int nbox) {
  int chosen = -1;
  for (int i = 0; i < nbox; ++i) {
    const int v = variant4(ctx[i]->kp);
    if (v < 0 || v > 3) return -1;
    if (chosen >= 0 && (v >> 1) != (chosen >> 1)) return -1;
    chosen = std::max(chosen, v);
  }
  return chosen;
}

bool multi4_eligible(erpp_ctx* const* ctx, int nbox) {
  if (nbox < 1 || multi4_variant(ctx, nbox) < 0) return false;
  for (int i = 0; i < nbox; ++i) {
    const erpp_kparams& kp = ctx[i]->kp;
    if (ctx[i]->fp64 || kp.design != 4 || kp.weights != ERPP_W_GAUSS || kp.kahan || kp.lag > 0 ||
        kp.full_force || !ctx[i]->entries || !ctx[i]->halo)
      return false;
  }
  return true;
}

template <int XM, int LMIN, int XW>
cudaError_t multi4_setup_kernels(Multi4* m, int nsm) {
  int nb = 0;
  cudaError_t e = cudaFuncSetAttribute(k_gather4_multi<XM, LMIN, XW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m->smem_g);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather4_multi<XM, LMIN, XW>, 256,
                                                      m->smem_g);
  m->grid_g = nsm * (nb > 0 ? nb : 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_scatter4_multi<XM, LMIN, XW>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m->smem_s);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter4_multi<XM, LMIN, XW>, 256,
                                                      m->smem_s);
  m->grid_s = nsm * (nb > 0 ? nb : 1);
  return e;
}

void multi4_destroy(Multi4* m) {
  if (!m) return;
  cudaFree(m->boxes);
  cudaFree(m->pboxes);
  cudaFree(m->items);
  cudaFree(m->pitems);
  cudaFree(m->counter);
  delete m;
}

// The descriptors of every box (their contexts' current buffers), the work
// items ordered by particles per tile (densest boxes first) and the counters.
cudaError_t multi4_create(erpp_ctx* const* ctx, const float* const* u, float* const* S,
                          const erpp_particles* parts, int nbox, Multi4** out) {
  *out = nullptr;
  Multi4* m = new Multi4();
  m->nbox = nbox;
  std::vector<BoxTiles> hb((size_t)nbox);
  std::vector<erpp_box_dev> hp((size_t)nbox);
  std::vector<int> order((size_t)nbox);
  std::vector<int64_t> npart((size_t)nbox);
  std::vector<int2> pitems;
  int64_t nitems = 0;
  for (int i = 0; i < nbox; ++i) {
    BoxTiles& d = hb[(size_t)i];
    memset(&d, 0, sizeof(d));
    const erpp_ctx* c = ctx[i];
    const erpp_particles& P = parts[i];
    npart[(size_t)i] = P.n;
    erpp_box_dev& q = hp[(size_t)i];
    memset(&q, 0, sizeof(q));
    q.kp = c->kp;
    q.n = P.n;
    q.cap = c->cap;
    q.ecap = c->entries_cap;
    q.ms = c->maxseg[0] * c->maxseg[1] * c->maxseg[2];
    q.nbins = nbins(c->kp);
    q.xw_len = c->xw_len;
    for (int a = 0; a < 3; ++a) {
      q.x[a] = P.x[a];
      q.v[a] = P.v[a];
      q.xp[a] = P.x_prev[a];
      q.D[a] = P.D[a];
    }
    q.radius = P.radius;
    q.rho_p = P.rho_p;
    q.geo_t = c->geo_t;
    q.geo_c = c->geo_c;
    q.d0x = c->d0x;
    q.tile_cnt = c->tile_cnt;
    q.tile_start = c->tile_start;
    q.piece_slot = c->piece_slot;
    q.entries = c->entries;
    q.up_part = c->up_part;
    q.fscat = c->fscat;
    q.S = S[i];
    q.halo = c->halo;
    q.err = c->err;
    for (int64_t f = 0; f < P.n; f += 256) pitems.push_back(make_int2(i, (int)f));
    d.kp = c->kp;
    d.use_tma = field_tensor_map(c->kp, u[i], &d.tmap) ? 1 : 0;
    d.u = u[i];
    d.S = S[i];
    d.halo = c->halo;
    d.start = c->tile_start;
    d.entries = c->entries;
    d.ecap = c->entries_cap;
    d.d0x = c->d0x;
    d.fscat = c->fscat;
    d.up_part = c->up_part;
    d.err = c->err;
    order[(size_t)i] = i;
    nitems += c->kp.ntiles;
    m->smem_g = std::max(m->smem_g, smem_bytes4(c->kp, 3, true));
    m->smem_s = std::max(m->smem_s, smem_bytes4(c->kp, 3, false));
  }
  if (nitems > (int64_t)1 << 30) {
    delete m;
    return cudaErrorInvalidValue;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)npart[(size_t)a] / ctx[a]->kp.ntiles >
           (double)npart[(size_t)b] / ctx[b]->kp.ntiles;
  });
  std::vector<int2> items;
  items.reserve((size_t)nitems);
  for (int i : order)
    for (int t = 0; t < ctx[i]->kp.ntiles; ++t) items.push_back(make_int2(i, t));
  m->nitems = (int)nitems;
  m->npitems = (int)pitems.size();
  m->variant = multi4_variant(ctx, nbox);
  cudaError_t e = cudaMalloc(&m->boxes, sizeof(BoxTiles) * (size_t)nbox);
  if (e == cudaSuccess) e = cudaMalloc(&m->pboxes, sizeof(erpp_box_dev) * (size_t)nbox);
  if (e == cudaSuccess) e = cudaMalloc(&m->items, sizeof(int2) * std::max<size_t>(items.size(), 1));
  if (e == cudaSuccess)
    e = cudaMalloc(&m->pitems, sizeof(int2) * std::max<size_t>(pitems.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&m->counter, 2 * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->boxes, hb.data(), sizeof(BoxTiles) * (size_t)nbox, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->pboxes, hp.data(), sizeof(erpp_box_dev) * (size_t)nbox,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(m->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pitems.empty())
    e = cudaMemcpy(m->pitems, pitems.data(), sizeof(int2) * pitems.size(),
                   cudaMemcpyHostToDevice);
  int dev = 0, nsm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    switch (m->variant) {
      case 0: e = multi4_setup_kernels<7, 6, 8>(m, nsm); break;
      case 1: e = multi4_setup_kernels<7, 5, 8>(m, nsm); break;
      case 2: e = multi4_setup_kernels<10, 9, 16>(m, nsm); break;
      default: e = multi4_setup_kernels<10, 8, 16>(m, nsm); break;
    }
  }
  if (e != cudaSuccess) {
    multi4_destroy(m);
    return e;
  }
  *out = m;
  return cudaSuccess;
}

template <int XM, int LMIN, int XW>
cudaError_t multi4_run(const Multi4* m, bool gather, cudaStream_t st) {
  if (gather)
    k_gather4_multi<XM, LMIN, XW><<<m->grid_g, 256, m->smem_g, st>>>(m->boxes, m->items,
                                                                      m->nitems, m->counter);
  else
    k_scatter4_multi<XM, LMIN, XW><<<m->grid_s, 256, m->smem_s, st>>>(m->boxes, m->items,
                                                                       m->nitems, m->counter + 1);
  return cudaGetLastError();
}

cudaError_t multi4_tiles(const Multi4* m, bool gather, cudaStream_t st) {
  switch (m->variant) {
    case 0: return multi4_run<7, 6, 8>(m, gather, st);
    case 1: return multi4_run<7, 5, 8>(m, gather, st);
    case 2: return multi4_run<10, 9, 16>(m, gather, st);
    default: return multi4_run<10, 8, 16>(m, gather, st);
  }
}

cudaError_t multi4_step(const Multi4* m, int first_step, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(m->counter, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = launch_bin_multi(m->pboxes, m->nbox, m->pitems, m->npitems, st);
  if (e == cudaSuccess) e = multi4_tiles(m, true, st);
  if (e == cudaSuccess) e = launch_advance_multi(m->pboxes, m->pitems, m->npitems, first_step, st);
  if (e == cudaSuccess) e = multi4_tiles(m, false, st);
  if (e == cudaSuccess && m->nitems > 0) {
    k_merge_rows_multi<<<m->nitems, kMergeThreads, 0, st>>>(m->boxes, m->items);
    k_merge_cols_multi<<<m->nitems, kMergeThreads, 0, st>>>(m->boxes, m->items);
    e = cudaGetLastError();
  }
  return e;
}


}  // namespace erpp
