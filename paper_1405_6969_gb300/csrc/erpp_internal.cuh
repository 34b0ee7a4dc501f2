// erpp_internal.cuh -- shared declarations of the ERPP CUDA library.
//
// Layout of the per-step data in HBM (FP32 tiled path):
//   geo_t[i]  float4  (t_x, t_y, t_z, pieces): fractional position of
//                     particle i inside its home cell; x/y-halo tiles: the
//                     number of pieces of its stencil (int bits)
//   geo_c[i]  int4    (c_x, c_y, c_z, pack): home cell and packed window
//                     (offset of the first node below the cell, window length)
//   xw[i]     float[XW] the particle's x-weights 2^(-beta_x d^2) over its
//                     x-window (zero beyond it), XW = 8 or 16
//   entries[] int4    one record per piece (particle, tile, periodic shift in
//                     y/z) whose window reaches the tile, grouped by tile and,
//                     inside a tile, by the bucket x0 mod 32 (counting sort):
//                     {particle, base | lx << 17 | ly << 22 | lz << 27,
//                      d0y bits, d0z bits}, base the shared-memory index of
//                     the piece's first node, d0 its distance (grid units)
//                     A particle belongs to the x-tile of its home cell and
//                     keeps its whole x-window there (tiles are staged with an
//                     x-halo); only y and z windows are cut at tile boundaries.
//   up_acc    float[3][n]  gathered velocity before normalisation (x-halo
//                     tiles); x/y-halo tiles instead keep each piece's sums
//                     in up_part[place of the piece's record], and
//                     piece_slot[k][n] holds the place of particle i's k-th
//                     piece once the binning is done
//   fscat[i]  float4  -(1/rho_f) D_i norm / dV, max|component|
//   d0x[i]    float   x/y-halo tiles: distance (grid units) from particle i
//                     to the first node of its x-window
//   halo      float   per tile, the scatter's x-halo columns (left hlo,
//                     right hhi), [tile][3][T_z][T_y][hlo + hhi]
// Grids are [3][nz][ny][nx] (x fastest).  Tiles: x-width W = 64 (last one
// ragged), T_y x T_z in y/z; a tile is staged in shared memory as
// [3][T_z][T_y][PX] with PX = 96 floats per row (a multiple of the 32 banks),
// local x' = x - (tile start - hlo).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/erpp.h"

// Weights of the coupling (erpp_kparams.weights).
#define ERPP_W_GAUSS 0  // the regularised Gaussian kernel, matching gather
#define ERPP_W_PIC 1    // trilinear projection and interpolation (cloud in cell)
#define ERPP_W_POINT 2  // Gaussian source, 4-point Lagrange point-value gather

// Sticky device error bits.
#define ERPP_ERRBIT_RANGE 1u
#define ERPP_ERRBIT_BOUNDS 2u
#define ERPP_ERRBIT_TIMEOUT 4u

// Packed window field of geo_c.w: bits 0-3 / 4-7 / 8-11 = -offset of the
// first window node from the home cell on x / y / z, bits 12-16 / 17-21 /
// 22-26 = window length on x / y / z, bit 31 = valid.
#define ERPP_GEO_VALID 0x80000000u

// Particle indices are 31-bit; the packed piece base is 17 bits.
#define ERPP_MAX_PARTICLES ((int64_t)0x7fffffff)
#define ERPP_BASE_BITS 17

// Kernel-side constants of one grid and parameter set.
struct erpp_kparams {
  int32_t n[3];      // nodes per axis
  int32_t T[3];      // tile size per axis (T[0] = W, the x-tile width)
  int32_t nt[3];     // tiles per axis
  int32_t ntiles;
  int32_t hlo;       // floor(c'): lowest window offset is -hlo (all axes)
  int32_t xs;        // longest window, floor(2 c') + 1 (all axes)
  int32_t xhlo, xhhi;// x-halo columns staged below / above a tile
  int32_t xlmin, xxs; // shortest / longest x-window (floor(2 c'_x), floor(2 c'_x) + 1)
  int32_t px, pxy;   // shared-memory pitches (floats) of one tile
  int32_t plane;     // floats per component of one tile = pxy * T_z
  int32_t design;    // 3: x-halo tiles, pieces cut in y and z (bucket bins);
                     // 4: x/y-halo tiles, pieces cut in z only, unit schedules
  int32_t yhlo, yhhi;// design 4: y-halo rows staged below / above a tile
  int32_t nthreads;  // design 4: threads per block of the tile kernels (256, 512)
  int32_t xoff;      // design 4: staged column of the tile's first node
                     // (xhlo rounded up to a multiple of 4)
  int64_t halo_per_tile; // design 4: floats of one tile's scatter halo strips
  int64_t ystrip_off;    // design 4: offset (floats) of the y-strips in them
  int32_t normalize, self_removal, kahan;
  int32_t weights;   // ERPP_W_GAUSS, ERPP_W_PIC or ERPP_W_POINT
  int32_t lag;       // ERPP_LAG: source delay in steps, round(eps_R / dt) >= 1; else 0
  int32_t full_force;// ERPP_FULL_FORCE
  int32_t xclip;     // design 4: x-windows cut at x-tile boundaries (no x-halo
                     // contributions, so no x-strips and no column merge)
  int32_t debug_stall;// test hook: after its copies land, the gather also waits
                      // on a barrier that nothing completes (the wait runs out)
  int64_t wait_ns;   // limit of every bounded device-side wait, nanoseconds
  double inv_dx[3];  // N / L
  double L[3];
  double cp[3];      // r_c / dx
  int cp_int[3];     // floor(cp)
  float cp_frac[3];  // cp - floor(cp), rounded to FP32
  float lap_k[3];    // dx_a^2 / sigma_R^4: scale of the weights' second
                     // derivatives in the particle position (general force)
  double dx[3];
  double dV;
  double rho_f, nu, eps_R, dt, mu;
  double gravity[3];
  double shear_rate;
  double raw_norm3;  // (2 pi sigma_R^2)^(-3/2)
  double raw_norm1;  // (2 pi sigma_R^2)^(-1/2)
  double self_pref64;// -(dt/rho_f) (2 pi self_s2)^(-3/2)
  double basset_c;   // 12 mu sqrt(pi / (nu dt)) (ERPP_FULL_FORCE; 0 when dt = 0)
  double sig2;       // sigma_R^2
  double self_s2;    // variance of the self disturbance as gathered
  float beta[3];     // log2(e) dx_a^2 / (2 sigma_R^2)
  float inv_rho_dV;  // 1 / (rho_f dV)
  float self_pref;   // -(dt/rho_f) (2 pi s2)^(-3/2)
  float self_inv_w;  // 1 / sqrt(2 s2)
  // float copies for the FP32 drag and increment of the advance
  float drag_f;      // 6 pi mu
  float rho_f_f;     // rho_f
  float dt_f;        // dt
  float grav_f[3];   // gravity
  float halfL_f[3];  // L / 2 (minimum-image pre-check)
  // bit patterns of 1e-4 L and (1 - 1e-4) L: a position strictly between them
  // needs no periodic wrap (non-negative doubles order as their bit patterns)
  int64_t wrap_lo_bits[3], wrap_hi_bits[3];
};

struct erpp_ctx {
  erpp_params params;
  erpp_kparams kp;
  int device;
  int fp64;
  int maxseg[3];          // most tiles one window can reach per axis
  int tile_req[3];        // requested T_y, T_z, threads of the x/y-halo tiles (0: default)
  int64_t wait_req_ns;    // erpp_debug_set_wait: bounded-wait limit (0: default)
  int stall_req;          // erpp_debug_set_wait: stall hook of the gather
  int scatter_mode;       // erpp_set_scatter_mode (ERPP_SCATTER_*)
  int cluster_probe;      // clustered scatter for the current tiling: 0 = not yet
                          // asked, 1 = resident clusters possible, 2 = not
  struct erpp_host_pipe* hp;  // erpp_step_host staging and streams (lazily created)
  int launches;           // kernels launched since erpp_step began (counted at each launch)
  int last_step_launches; // kernels the most recent erpp_step launched
  // scratch (owned)
  int64_t cap;            // particle capacity of the per-particle arrays
  float4* geo_t;
  int4* geo_c;
  float* xw;              // [cap][xw_len] x-weights per particle (x-halo tiles)
  float* d0x;             // [cap] x/y-halo tiles: x-distance of the window's first node
  float4* lapc;           // [2 cap] general force, x/y-halo tiles: per particle the mean
                          // and variance of its window offsets under the weights,
                          // (mu_x, V_x, mu_y, V_y), (mu_z, V_z, 0, 0)
  float4* lap_part;       // [entries_cap] general force: each piece's Laplacian sums
  int xw_len;
  float* up_acc;          // [3][cap] gathered velocity (x-halo tiles cut in y and z)
  float4* up_part;        // [entries_cap] x/y-halo tiles: each piece's gathered sums,
                          // at its place in the piece records
  float4* fscat;
  double* up64;           // FP64 mode or other weights: gathered velocity [3][cap]
  int32_t* w_key;         // other weights: sort key, place and order of each particle [cap]
  int32_t* w_slot;
  int32_t* w_perm;
  int32_t* w_cnt;         // [w_nbins]: particles per cell block (last: invalid positions)
  int32_t* w_start;       // [w_nbins + 1]
  int32_t* w_tmp;         // scan chunk totals
  int w_nbins;
  double* lag_ring;       // ERPP_LAG: [lag + 1][6][cap] positions and forces of past steps
  int64_t lag_step;       // steps since the last first_step
  int64_t lag_n;          // particle count of those steps
  double* ff_lap;         // ERPP_FULL_FORCE: gathered Laplacian [3][cap]
  double* ff_prev;        // ERPP_FULL_FORCE: u~ and lap u~ of the previous step [6][cap]
  int64_t ff_n;           // particle count since the last first step (-1: none)
  int4* entries;
  int64_t entries_cap;
  float* halo;            // scatter x-halo columns, [ntiles][3][T_z][T_y][xhlo + xhhi]
  int32_t* tile_cnt;      // [32 ntiles]: pieces per (tile, bucket) bin
  int32_t* tile_start;    // [32 ntiles + 1]
  int32_t* piece_slot;    // [maxseg product][cap]: each piece's place in its bin
  int32_t* scan_tmp;      // [ceil(32 ntiles / 4096)] chunk totals of the scan
  uint32_t* err;          // device error word
  double* red;            // reduction scratch
  int red_cap;
  // per-phase timing (erpp_profile_*)
  int prof_on;
  int prof_n;             // event sets recorded since the last read
  cudaEvent_t* prof_ev;   // [kProfSets][5]
};

constexpr int kProfSets = 1024;
// Default limit of a bounded device-side wait (a staged tile's copies land
// within microseconds; the limit only guards against a copy that never does).
constexpr int64_t kDefaultWaitNs = 250000000;

// Where the FP32 tile gather leaves its sums (see the layout above).
struct erpp_acc {
  const float* up_acc;      // x-halo tiles: [3][stride]
  int64_t stride;
  const float4* up_part;    // x/y-halo tiles: per piece
  const int32_t* piece_slot;// [k][n]: place of particle i's k-th piece
  int64_t n;
};

// One box of the multi-box launches (batched boxes): its kernel parameters,
// sizes, and the buffers of its context and particle state, in device memory.
struct erpp_box_dev {
  erpp_kparams kp;
  int64_t n;      // particles
  int64_t cap;    // particle capacity of the context's arrays (their stride)
  int64_t ecap;   // piece-record capacity
  int32_t ms;     // most pieces per particle
  int32_t nbins;  // tiles
  int32_t xw_len; // longest x-window the binning accepts
  double* x[3];
  double* v[3];
  double* xp[3];
  double* D[3];
  const double* radius;
  const double* rho_p;
  float4* geo_t;
  int4* geo_c;
  float* d0x;
  int32_t* tile_cnt;
  int32_t* tile_start;
  int32_t* piece_slot;
  int4* entries;
  float4* up_part;
  float4* fscat;
  float* S;
  float* halo;
  uint32_t* err;
};

// ---- host-side launchers (stream-ordered, no synchronisation) ----
namespace erpp {
// Multi-box launches over pitems = (box, first particle) chunks of 256
// particles or the boxes themselves: the binning (counts cleared, counted,
// scanned per box, records filled: four launches) and the advance.
cudaError_t launch_bin_multi(const erpp_box_dev* boxes, int nbox, const int2* pitems,
                             int npitems, cudaStream_t st);
cudaError_t launch_advance_multi(const erpp_box_dev* boxes, const int2* pitems, int npitems,
                                 int first_step, cudaStream_t st);

erpp_status derive_ctx(const erpp_params* p, erpp_ctx* c);
erpp_status ensure_capacity(erpp_ctx* c, int64_t n);  // may allocate (synchronous)
int xw_len(const erpp_kparams& kp);
inline int nbins(const erpp_kparams& kp) { return kp.design == 4 ? kp.ntiles : kp.ntiles * 32; }
// The coupling step of erpp_step (arguments already checked); records
// after_advance (when not null) on st once the particles are advanced.
erpp_status step_device(erpp_ctx* c, const void* u, const erpp_particles* P, void* S,
                        int first_step, cudaStream_t st, cudaEvent_t after_advance);
// The source of forces D at positions x into S (zeroed first), -(1/rho_f) times
// the context's projection weights.
cudaError_t scatter_source(erpp_ctx* c, int64_t n, const double* const x[3],
                           const double* const D[3], void* S, cudaStream_t st);
// Frees the host-data pipeline of erpp_step_host (synchronises the device).
void free_host_pipe(erpp_ctx* c);
cudaError_t bin_particles(erpp_ctx* ctx, int64_t n, const double* const x[3], bool zero_acc,
                          cudaStream_t st);
cudaError_t launch_gather_f32(erpp_ctx* ctx, const float* u, int64_t n, cudaStream_t st);
cudaError_t launch_scatter_f32(erpp_ctx* ctx, float* S, cudaStream_t st);  // + x-halo merge
cudaError_t launch_gather_f32_4(erpp_ctx* ctx, const float* u, cudaStream_t st);
// General force on x/y-halo tiles: the gather of the velocity and of its
// Laplacian (per-piece sums in up_part and lap_part), and their per-particle
// totals: up = norm * sum + shear y (x component), lap = norm * sum.
cudaError_t launch_gather_lap_f32_4(erpp_ctx* ctx, const float* u, cudaStream_t st);
cudaError_t launch_finalize_full(erpp_ctx* ctx, int64_t n, const double* const x[3],
                                 double* const up[3], double* lap, int64_t lap_stride,
                                 cudaStream_t st);
size_t smem_bytes4(const erpp_kparams& kp, int copies, bool gather);
// Batch width of the x/y-halo tile kernels: 8 for x-windows of at most 7
// nodes, else 16 (256 or 128 pieces per batch).
int xw4(const erpp_kparams& kp);
cudaError_t launch_scatter_f32_4(erpp_ctx* ctx, float* S, cudaStream_t st);  // + halo merge
// Many boxes (batched) in one gather launch and one scatter launch: persistent
// blocks pull (box, tile) items, densest boxes first, from a counter.  Needs
// every box on x/y-halo tiles, FP32, Gaussian weights, the fixed-point
// scatter and the same window variant (multi4_eligible).  The descriptors
// hold the contexts' buffers as they are at creation.
struct Multi4;
bool multi4_eligible(erpp_ctx* const* ctx, int nbox);
cudaError_t multi4_create(erpp_ctx* const* ctx, const float* const* u, float* const* S,
                          const erpp_particles* parts, int nbox, Multi4** out);
// The coupling step of every box in ten launches: binning (4), gather,
// advance, scatter and the two halo merges of all boxes, and the clearing of
// the work counters.
cudaError_t multi4_step(const Multi4* m, int first_step, cudaStream_t st);
void multi4_destroy(Multi4* m);

cudaError_t launch_finalize_up(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               double* const up[3], cudaStream_t st);
// fscat_i = scale * norm_i * D_i (scale = -1/(rho_f dV) for the source).
cudaError_t launch_prep_fscat(erpp_ctx* ctx, int64_t n, const double* const D[3], float scale,
                              cudaStream_t st);
// xs, Ds (optional): position and force of the source whose disturbance is
// removed, instead of P's x_prev and D.
cudaError_t launch_advance(erpp_ctx* ctx, const erpp_particles* P, const double* const up[3],
                           bool from_acc, bool write_fscat, int first_step, cudaStream_t st,
                           const double* const xs[3] = nullptr,
                           const double* const Ds[3] = nullptr);
// ERPP_FULL_FORCE: gathered velocity (plus the mean shear) and its Laplacian in
// the particle position, into up and ctx->ff_lap; then the general-force
// advance from them (ctx->ff_prev holds u~ and lap u~ of the previous step).
cudaError_t launch_gather_faxen(erpp_ctx* ctx, const void* u, int64_t n,
                                const double* const x[3], double* const up[3], cudaStream_t st);
cudaError_t launch_advance_full(erpp_ctx* ctx, const erpp_particles* P,
                                const double* const up[3], int first_step, cudaStream_t st);
// ring[slot] <- (x, D) for the delayed source (slot: six arrays of ctx->cap doubles).
cudaError_t launch_lag_store(erpp_ctx* ctx, int64_t n, const double* const x[3],
                             const double* const D[3], double* slot, cudaStream_t st);
cudaError_t launch_gather_f64(erpp_ctx* ctx, const double* u, int64_t n,
                              const double* const x[3], double* const up[3], cudaStream_t st);
cudaError_t launch_scatter_f64(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               const double* const D[3], double fscale, double* S,
                               cudaStream_t st);
// Per particle: outv = alpha sum_j F_j W (if outv), outx = alpha sum_j (F_j . v)
// dW/dx + shear_coef v_x on y.
cudaError_t launch_adjoint(erpp_ctx* ctx, int64_t n, const double* const x[3], const void* F,
                           const double* const v[3], double alpha, double shear_coef,
                           double* const outv[3], double* const outx[3], cudaStream_t st);
cudaError_t launch_momentum(erpp_ctx* ctx, const void* S, int64_t n, const double* const x[3],
                            const double* const D[3], cudaStream_t st);
cudaError_t launch_windows(erpp_ctx* ctx, int64_t n, const double* const x[3], int32_t* jlo,
                           int32_t* jhi, cudaStream_t st);
// Other weights (ERPP_W_PIC, ERPP_W_POINT): the gather of u (the context's grid
// type) into up, and the PIC source S = fscale sum_p D_p w_p(j) / dV (zeroes S
// first).
// Exclusive scan of cnt[0..nbins) into start[0..nbins] (start[nbins] = total);
// tmp holds nbins / 4096 + 1 ints.
cudaError_t launch_scan(erpp_ctx* ctx, const int32_t* cnt, int32_t* start, int32_t* tmp,
                        int nbins, cudaStream_t st);
// Other weights: orders the particles by 8 x 8 x 8-node block of their cell
// (counting sort into ctx->w_perm), so that the gathers and the PIC source
// walk the grid block by block.
cudaError_t sort_by_cell_block(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               cudaStream_t st);
cudaError_t launch_gather_weights(erpp_ctx* ctx, const void* u, int64_t n,
                                  const double* const x[3], double* const up[3], cudaStream_t st);
cudaError_t launch_scatter_pic(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               const double* const D[3], double fscale, void* S,
                               cudaStream_t st);

}  // namespace erpp

// ---- device helpers shared by the kernels ----

// Window of one coordinate, exactly as the oracle decides it: s = x * (N/L)
// rounded once, j_lo = ceil(s - c'), j_hi = floor(s + c') with one rounding
// each (no contraction into fused multiply-adds).
__device__ __forceinline__ void erpp_axis_window(double x, double inv_dx, double cp, double* s,
                                                 double* jlo, double* jhi) {
  double sv = __dmul_rn(x, inv_dx);
  *s = sv;
  *jlo = ceil(__dadd_rn(sv, -cp));
  *jhi = floor(__dadd_rn(sv, cp));
}

// Exact FP32 -> FP64 and round-to-nearest-even FP64 -> FP32 conversions by
// integer operations on the bit patterns.  The hardware conversions run on
// the FP64 pipe, which is narrow on this GPU (about 1.5 operations per clock
// per SM, so every FP64-pipe instruction per particle costs about 2 us over a
// million particles); these give the same results with integer instructions.
// Zero, subnormal, infinite and NaN inputs, and results outside the normal
// FP32 range, branch to the hardware conversion.
static __device__ __noinline__ double erpp_f2d_hw(float f) { return (double)f; }
static __device__ __noinline__ float erpp_d2f_hw(double x) { return (float)x; }
__device__ __forceinline__ double erpp_f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return erpp_f2d_hw(f);
  const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                               ((unsigned long long)(e + (1023u - 127u)) << 52) |
                               ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}
__device__ __forceinline__ float erpp_d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu) - (1023 - 127);  // biased FP32 exponent
  if (e <= 0 || e >= 255) return erpp_d2f_hw(x);
  const unsigned mh = (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rem = (unsigned)(b & 0x1fffffffu);
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u))) ? 1u : 0u;
  return __uint_as_float(((((unsigned)(b >> 63)) << 31) | ((unsigned)e << 23) | mh) + up);
}

// The window of one axis as the binning uses it: s = x N/L (FP64, one
// rounding), the home cell ci = floor(s), jlo = ceil(RN(s - cp)),
// jhi = floor(RN(s + cp)) and t = RN_f32(s - ci), which are the values of
// the FP64 form above (each rounding done once).  Only the product is taken
// in FP64: the FP64 pipe is narrow, so the rest is integer and FP32 work.
// With s = ci + f and cp = ck + cf (integer and fractional parts), s - cp =
// (ci - ck) + (f - cf) and s + cp = (ci + ck) + (f + cf); f is read exactly
// from the bits of s, and the FP32 estimates of g = f - cf and h = f + cf
// (error below 2e-7) decide the ceiling and floor wherever they are farther
// than 1e-5 from the points where the rounding of the sum could move the
// result (g near -1 or 0, h near 1 or 2).  Elsewhere, and for s below 2^-126
// in fraction, the FP64 form runs.
struct erpp_axis_win {
  int ci, lo, hi;
  float t;
};
__device__ __forceinline__ erpp_axis_win erpp_axis_window_lean(double x, double inv_dx, double cp,
                                                               int ck, float cf) {
  erpp_axis_win w;
  const double s = __dmul_rn(x, inv_dx);
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  const int ef = (int)((b >> 52) & 0x7ffu);
  bool lean = ef != 0 && (b >> 63) == 0ull;
  if (lean) {
    // s = m 2^-sh, m with its implicit bit
    const int sh = 1075 - ef;
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int ci = sh < 64 ? (int)(m >> sh) : 0;
    const unsigned long long fb = sh < 64 ? (m & ((1ull << sh) - 1ull)) : m;  // f = fb 2^-sh
    float t = 0.f;
    if (fb != 0ull) {
      const int lz = __clzll((long long)fb);
      const int E = (63 - lz) - sh + 127;  // biased FP32 exponent of f
      const unsigned long long mm = fb << lz;
      const unsigned int hi24 = (unsigned int)(mm >> 40);
      const unsigned long long rem = mm & ((1ull << 40) - 1ull);
      const unsigned int up =
          (rem > (1ull << 39) || (rem == (1ull << 39) && (hi24 & 1u))) ? 1u : 0u;
      lean = E >= 1;
      t = __uint_as_float(((unsigned int)max(E, 0) << 23) + (hi24 - (1u << 23)) + up);
    }
    const float g = t - cf, h = t + cf;
    lean = lean && fabsf(g) > 1e-5f && g > -1.f + 1e-5f && fabsf(h - 1.f) > 1e-5f &&
           h < 2.f - 1e-5f;
    w.ci = ci;
    w.lo = ci - ck + (g > 0.f ? 1 : 0);
    w.hi = ci + ck + (h > 1.f ? 1 : 0);
    w.t = t;
  }
  if (!lean) {
    w.ci = __double2int_rd(s);
    w.lo = __double2int_ru(__dadd_rn(s, -cp));
    w.hi = __double2int_rd(__dadd_rn(s, cp));
    w.t = __double2float_rn(__dadd_rn(s, -(double)w.ci));
  }
  return w;
}

__device__ __forceinline__ int erpp_geo_off(uint32_t pack, int a) {
  return -(int)((pack >> (4 * a)) & 15u);
}
__device__ __forceinline__ int erpp_geo_nw(uint32_t pack, int a) {
  return (int)((pack >> (12 + 5 * a)) & 31u);
}

__device__ __forceinline__ void erpp_set_err(uint32_t* err, uint32_t bit) {
  if (err) atomicOr(err, bit);
}

// Programmatic dependent launch between the kernels of a step.  Each such
// kernel calls erpp_pdl_enter() before touching global memory: it lets the
// next kernel on the stream be launched once every block of this one has
// started, then waits until the previous kernel has completed and its writes
// are visible.  A kernel launched without the attribute returns from the wait
// at once.  The next kernel's blocks, once resident, wait in hardware (no
// polling), and they are only launched after every block of this kernel is
// resident or done, so no block waits for one that cannot run.
__device__ __forceinline__ void erpp_pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launches kern on st with programmatic stream serialisation (the kernel
// must call erpp_pdl_enter() first) and, when cluster_x > 0, clusters of
// cluster_x blocks along x.
template <typename... P, typename... A>
inline cudaError_t erpp_launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t st, unsigned cluster_x, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  int na = 0;
  at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[na].val.programmaticStreamSerializationAllowed = 1;
  ++na;
  if (cluster_x > 0) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = cluster_x;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// Kernel normalisation of one particle from its geometry record: the gather
// returns norm * sum_j e_x e_y e_z u_j with e_a = 2^(-beta_a d_a^2) (d in grid
// units), so norm = 1 / (sum_x e_x sum_y e_y sum_z e_z) for unit discrete mass
// per axis, or dV (2 pi sigma_R^2)^(-3/2) for the raw Gaussian.
__device__ __forceinline__ float erpp_norm(const erpp_kparams& kp, float4 gt, int4 gc) {
  if (!kp.normalize) return (float)(kp.dV * kp.raw_norm3);
  const uint32_t pack = (uint32_t)gc.w;
  if (!(pack & ERPP_GEO_VALID)) return 0.f;
  const float t[3] = {gt.x, gt.y, gt.z};
  float prod = 1.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int nw = (int)((pack >> (12 + 5 * a)) & 31u);
    const float d0 = -(float)((pack >> (4 * a)) & 15u) - t[a];
    float sum = 0.f;
    for (int k = 0; k < nw; ++k) {
      const float d = d0 + (float)k;
      sum += exp2f(-kp.beta[a] * d * d);
    }
    prod *= sum;
  }
  return 1.f / prod;
}

// Per axis, the mean mu and variance V of the offsets u = node - particle
// (grid units) of the particle's window under its weights e(u) =
// 2^(-beta u^2).  The second derivative in the particle position of the
// normalised weight e / sum e is then e / sum e * lap_k ((u - mu)^2 - V)
// (differentiate the quotient twice: the normalising sum contributes the
// mean and variance terms); for the raw Gaussian, mu = 0 and V = sigma_R^2
// in grid units.  out: (mu_x, V_x, mu_y, V_y), (mu_z, V_z, 0, 0).
__device__ __forceinline__ void erpp_lap_moments(const erpp_kparams& kp, const float t[3],
                                                 const int off[3], const int nw[3],
                                                 float4 out[2]) {
  float m[3], v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!kp.normalize) {
      m[a] = 0.f;
      v[a] = 1.4426950408889634f / (2.f * kp.beta[a]);
      continue;
    }
    const float d0 = (float)off[a] - t[a];
    float s = 0.f, s1 = 0.f, s2 = 0.f;
    for (int k = 0; k < nw[a]; ++k) {
      const float d = d0 + (float)k;
      const float e = exp2f(-kp.beta[a] * d * d);
      s += e;
      s1 = fmaf(e, d, s1);
      s2 = fmaf(e * d, d, s2);
    }
    const float inv = 1.f / s;
    m[a] = s1 * inv;
    v[a] = fmaf(-m[a], m[a], s2 * inv);
  }
  out[0] = make_float4(m[0], v[0], m[1], v[1]);
  out[1] = make_float4(m[2], v[2], 0.f, 0.f);
}

// The gathered sums of particle i (before normalisation): x/y-halo tiles add
// the sums of its pieces in piece order (deterministic), x-halo tiles read
// the atomically accumulated sums.
__device__ __forceinline__ void erpp_gathered(const erpp_kparams& kp, const erpp_acc& acc,
                                              float4 gt, int64_t i, float out[3]) {
  if (kp.design == 4) {
    const int np = __float_as_int(gt.w);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    // four pieces at a time: their places, then their sums, are loaded
    // together (independent loads in flight at once), then added in order
    for (int k0 = 0; k0 < np; k0 += 4) {
      int sl[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        sl[j] = k0 + j < np ? acc.piece_slot[(int64_t)(k0 + j) * acc.n + i] : -1;
      float4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        v[j] = sl[j] >= 0 ? acc.up_part[sl[j]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (k0 + j < np) {
          a0 += v[j].x;
          a1 += v[j].y;
          a2 += v[j].z;
        }
      }
    }
    out[0] = a0;
    out[1] = a1;
    out[2] = a2;
  } else {
    out[0] = acc.up_acc[i];
    out[1] = acc.up_acc[acc.stride + i];
    out[2] = acc.up_acc[2 * acc.stride + i];
  }
}

__device__ __forceinline__ int erpp_floordiv(int a, int n) {
  int q = a / n;
  return (a % n != 0 && ((a < 0) != (n < 0))) ? q - 1 : q;
}
