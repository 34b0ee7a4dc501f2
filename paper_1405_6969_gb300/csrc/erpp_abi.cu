// erpp_abi.cu -- the C ABI: parameter validation, context and scratch
// management, and the stream-ordered launch sequences of each entry point
// (the step with the regularised kernel, with other weights, with the
// delayed source and with the general force).
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "erpp_internal.cuh"

namespace {

const double kPi = 3.141592653589793238462643;

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Most (tile, image) pieces a window of up to `xs` nodes can be cut into on
// one axis, found by trying every window start.
int max_pieces(int n, int T, int hlo, int xs) {
  int best = 1;
  for (int jlo = -hlo; jlo < n + 1; ++jlo) {
    int cnt = 0;
    for (int j = jlo; j <= jlo + xs - 1;) {
      int m = (j >= 0) ? j / n : -((-j + n - 1) / n);
      int w = j - m * n;
      int t = w / T;
      int e = std::min(std::min((t + 1) * T, n) - w + j - 1, jlo + xs - 1);
      ++cnt;
      j = e + 1;
    }
    best = std::max(best, cnt);
  }
  return best;
}

erpp_status set_cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return ERPP_OK;
  if (e == cudaErrorMemoryAllocation) return ERPP_ENOMEM;
  return ERPP_ECUDA;
}

void free_scratch(erpp_ctx* c) {
  cudaFree(c->geo_t);
  cudaFree(c->geo_c);
  cudaFree(c->xw);
  cudaFree(c->up_acc);
  cudaFree(c->up_part);
  cudaFree(c->d0x);
  cudaFree(c->lapc);
  cudaFree(c->lap_part);
  c->up_part = nullptr;
  c->d0x = nullptr;
  c->lapc = nullptr;
  c->lap_part = nullptr;
  cudaFree(c->fscat);
  cudaFree(c->entries);
  cudaFree(c->piece_slot);
  cudaFree(c->up64);
  cudaFree(c->w_key);
  cudaFree(c->w_slot);
  cudaFree(c->w_perm);
  c->w_key = c->w_slot = c->w_perm = nullptr;
  cudaFree(c->lag_ring);
  c->lag_ring = nullptr;
  cudaFree(c->ff_lap);
  cudaFree(c->ff_prev);
  c->ff_lap = c->ff_prev = nullptr;
  c->geo_t = nullptr;
  c->geo_c = nullptr;
  c->xw = nullptr;
  c->up_acc = nullptr;
  c->fscat = nullptr;
  c->entries = nullptr;
  c->piece_slot = nullptr;
  c->up64 = nullptr;
  c->cap = 0;
  c->entries_cap = 0;
}

}  // namespace

namespace erpp {

// Grow the per-particle scratch to hold n particles (synchronous when it
// grows; the device allocation waits for outstanding work).
erpp_status ensure_capacity(erpp_ctx* c, int64_t n) {
  if (n <= c->cap) return ERPP_OK;
  int64_t cap = std::max<int64_t>(n, 1024);
  free_scratch(c);
  // the step histories (delayed source, general force) lived in the scratch:
  // the next step of such a context must be a first step
  c->lag_n = -1;
  c->ff_n = -1;
  cudaError_t e = cudaSuccess;
  if (c->fp64 || c->kp.weights != ERPP_W_GAUSS)
    e = cudaMalloc(&c->up64, sizeof(double) * 3 * (size_t)cap);
  if (c->kp.full_force && e == cudaSuccess) {
    e = cudaMalloc(&c->ff_lap, sizeof(double) * 3 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->ff_prev, sizeof(double) * 6 * (size_t)cap);
    if (e == cudaSuccess && !c->up64) e = cudaMalloc(&c->up64, sizeof(double) * 3 * (size_t)cap);
  }
  if (c->kp.lag > 0 && e == cudaSuccess)
    e = cudaMalloc(&c->lag_ring, sizeof(double) * 6 * (size_t)cap * (size_t)(c->kp.lag + 1));
  if (c->kp.weights != ERPP_W_GAUSS || (c->kp.full_force && !c->fp64)) {
    if (e == cudaSuccess) e = cudaMalloc(&c->w_key, sizeof(int32_t) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->w_slot, sizeof(int32_t) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->w_perm, sizeof(int32_t) * (size_t)cap);
  }
  if (!c->fp64 && e == cudaSuccess) {
    int64_t ecap = cap * (int64_t)c->maxseg[0] * c->maxseg[1] * c->maxseg[2];
    e = cudaMalloc(&c->geo_t, sizeof(float4) * (size_t)cap);
    if (e == cudaSuccess && c->kp.design != 4)
      e = cudaMalloc(&c->xw, sizeof(float) * (size_t)c->xw_len * (size_t)cap);
    if (e == cudaSuccess && c->kp.design == 4) e = cudaMalloc(&c->d0x, sizeof(float) * (size_t)cap);
    if (e == cudaSuccess && c->kp.design == 4 && c->kp.full_force)
      e = cudaMalloc(&c->lapc, 2 * sizeof(float4) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->geo_c, sizeof(int4) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->up_acc, sizeof(float) * 3 * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->fscat, sizeof(float4) * (size_t)cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->entries, sizeof(int4) * (size_t)ecap);
    if (e == cudaSuccess && c->kp.design == 4)
      e = cudaMalloc(&c->up_part, sizeof(float4) * (size_t)ecap);
    if (e == cudaSuccess && c->kp.design == 4 && c->kp.full_force)
      e = cudaMalloc(&c->lap_part, sizeof(float4) * (size_t)ecap);
    if (e == cudaSuccess) e = cudaMalloc(&c->piece_slot, sizeof(int32_t) * (size_t)ecap);
    c->entries_cap = ecap;
  }
  if (e != cudaSuccess) {
    free_scratch(c);
    return set_cuda_err(e);
  }
  c->cap = cap;
  return ERPP_OK;
}

}  // namespace erpp

namespace {

bool valid_vec(const double* const v[3]) { return v && v[0] && v[1] && v[2]; }

// Tile tables and scatter halo of the FP32 path, for the context's geometry.
erpp_status alloc_tile_tables(erpp_ctx* c) {
  if (c->fp64) return ERPP_OK;
  const erpp_kparams& kp = c->kp;
  const size_t nbins = (size_t)erpp::nbins(kp);
  cudaError_t e = cudaMalloc(&c->tile_cnt, sizeof(int32_t) * nbins);
  if (e == cudaSuccess) e = cudaMalloc(&c->tile_start, sizeof(int32_t) * (nbins + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->scan_tmp, sizeof(int32_t) * (nbins / 4096 + 1));
  const size_t hb = (size_t)kp.ntiles * (size_t)kp.halo_per_tile;
  if (e == cudaSuccess) e = cudaMalloc(&c->halo, sizeof(float) * hb);
  return set_cuda_err(e);
}

void free_tile_tables(erpp_ctx* c) {
  cudaFree(c->tile_cnt);
  cudaFree(c->tile_start);
  cudaFree(c->scan_tmp);
  cudaFree(c->halo);
  c->tile_cnt = c->tile_start = c->scan_tmp = nullptr;
  c->halo = nullptr;
}

// Cell-block tables of the other weights' particle sort (8 x 8 x 8-node blocks
// plus one bin for invalid positions).
erpp_status alloc_weight_tables(erpp_ctx* c) {
  if (c->kp.weights == ERPP_W_GAUSS && !(c->kp.full_force && !c->fp64)) return ERPP_OK;
  const erpp_kparams& kp = c->kp;
  int64_t nb = 1;
  for (int a = 0; a < 3; ++a) nb *= (kp.n[a] + 7) / 8;
  if (nb + 1 > (int64_t)1 << 30) return ERPP_EINVAL;
  c->w_nbins = (int)nb + 1;
  cudaError_t e = cudaMalloc(&c->w_cnt, sizeof(int32_t) * (size_t)c->w_nbins);
  if (e == cudaSuccess) e = cudaMalloc(&c->w_start, sizeof(int32_t) * ((size_t)c->w_nbins + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->w_tmp, sizeof(int32_t) * (c->w_nbins / 4096 + 1));
  return set_cuda_err(e);
}

erpp_status check_n(int64_t n) {
  if (n < 0 || n > ERPP_MAX_PARTICLES) return ERPP_EINVAL;
  return ERPP_OK;
}

}  // namespace

extern "C" {

const char* erpp_status_string(erpp_status s) {
  switch (s) {
    case ERPP_OK: return "ok";
    case ERPP_EINVAL: return "invalid argument";
    case ERPP_ENOMEM: return "device allocation failed";
    case ERPP_ECUDA: return "CUDA runtime error";
    case ERPP_ERANGE: return "particle position NaN/Inf or outside the box";
    case ERPP_EBOUNDS: return "internal capacity or index check failed";
    case ERPP_ETIMEOUT: return "bounded device wait gave up";
    case ERPP_ESTATE: return "call not valid in the current state";
  }
  return "unknown status";
}

}  // extern "C"

namespace erpp {

// Validates the parameters and fills the context's derived constants (kernel
// parameters, tile geometry, piece bounds).  Host only: no CUDA call, no
// allocation.
erpp_status derive_ctx(const erpp_params* p, erpp_ctx* c) {
  if (!p || !c) return ERPP_EINVAL;
  const int n[3] = {p->nx, p->ny, p->nz};
  const double L[3] = {p->Lx, p->Ly, p->Lz};
  for (int a = 0; a < 3; ++a)
    if (n[a] < 1 || n[a] > (1 << 20) || !finite_pos(L[a])) return ERPP_EINVAL;
  if (!finite_pos(p->nu) || !finite_pos(p->rho_f) || !finite_pos(p->eps_R) ||
      !finite_pos(p->cutoff) || !isfinite(p->dt) || p->dt < 0.0 || !isfinite(p->shear_rate))
    return ERPP_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->gravity[a])) return ERPP_EINVAL;
  const uint32_t prec = p->flags & (ERPP_FP32 | ERPP_FP64);
  if (prec != ERPP_FP32 && prec != ERPP_FP64) return ERPP_EINVAL;
  if ((p->flags & ERPP_KAHAN) && prec != ERPP_FP32) return ERPP_EINVAL;
  if (p->flags & ~(uint32_t)(ERPP_FP32 | ERPP_FP64 | ERPP_NORMALIZE | ERPP_SELF_REMOVAL |
                             ERPP_KAHAN | ERPP_PIC | ERPP_POINT_GATHER | ERPP_LAG |
                             ERPP_FULL_FORCE))
    return ERPP_EINVAL;
  if ((p->flags & ERPP_LAG) && ((p->flags & (ERPP_PIC | ERPP_POINT_GATHER)) || !(p->dt > 0.0) ||
                                !(p->eps_R / p->dt < 1.0e6)))
    return ERPP_EINVAL;
  if ((p->flags & ERPP_FULL_FORCE) &&
      ((p->flags & (ERPP_PIC | ERPP_POINT_GATHER | ERPP_LAG)) || !(p->dt > 0.0)))
    return ERPP_EINVAL;
  if ((p->flags & ERPP_PIC) &&
      (p->flags & (ERPP_POINT_GATHER | ERPP_SELF_REMOVAL | ERPP_KAHAN)))
    return ERPP_EINVAL;
  if ((double)n[0] * n[1] * n[2] * 3.0 >= 9.0e18) return ERPP_EINVAL;

  erpp_kparams kp;
  memset(&kp, 0, sizeof(kp));
  // Same expressions, same order as the FP64 oracle: the stencil windows
  // must agree bit for bit.
  const double sig2 = (2.0 * p->nu) * p->eps_R;
  const double sig = sqrt(sig2);
  const double rc = p->cutoff * sig;
  double cpmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    kp.n[a] = n[a];
    kp.L[a] = L[a];
    kp.inv_dx[a] = (double)n[a] / L[a];
    kp.dx[a] = L[a] / (double)n[a];
    kp.cp[a] = rc * kp.inv_dx[a];
    kp.cp_int[a] = (int)floor(kp.cp[a]);
    kp.cp_frac[a] = (float)(kp.cp[a] - floor(kp.cp[a]));
    if (!(2.0 * rc < L[a])) return ERPP_EINVAL;
    cpmax = std::max(cpmax, kp.cp[a]);
  }
  double cpmin = std::min(kp.cp[0], std::min(kp.cp[1], kp.cp[2]));
  if (cpmin < 1.0) return ERPP_EINVAL;  // r_c must reach at least one grid spacing
  // A window starts at most floor(c') nodes below the particle's cell and holds
  // at most floor(2 c') + 1 nodes (one more when 2 c' sits within rounding of
  // an integer).
  kp.hlo = (int)floor(cpmax);
  kp.xs = (int)floor(2.0 * cpmax + 1e-6) + 1;
  if (kp.hlo > 15 || kp.xs > 31) return ERPP_EINVAL;  // windows of at most 31 nodes
  kp.dV = kp.dx[0] * kp.dx[1] * kp.dx[2];
  kp.rho_f = p->rho_f;
  kp.nu = p->nu;
  kp.eps_R = p->eps_R;
  kp.dt = p->dt;
  kp.mu = p->rho_f * p->nu;
  for (int a = 0; a < 3; ++a) kp.gravity[a] = p->gravity[a];
  kp.shear_rate = p->shear_rate;
  kp.sig2 = sig2;
  kp.raw_norm3 = pow(2.0 * kPi * sig2, -1.5);
  kp.lag = (p->flags & ERPP_LAG) ? std::max(1, (int)lround(p->eps_R / p->dt)) : 0;
  kp.full_force = (p->flags & ERPP_FULL_FORCE) ? 1 : 0;
  kp.wait_ns = c->wait_req_ns > 0 ? c->wait_req_ns : kDefaultWaitNs;
  kp.debug_stall = c->stall_req ? 1 : 0;
  kp.weights = (p->flags & ERPP_PIC) ? ERPP_W_PIC
               : (p->flags & ERPP_POINT_GATHER) ? ERPP_W_POINT : ERPP_W_GAUSS;
  // The disturbance as the gather sees it: forcing diffused one step, plus the
  // matching kernel's own sigma_R^2 (none for a point-value gather).
  kp.self_s2 = (2.0 * p->nu) * (p->eps_R + p->dt) +
               (kp.weights == ERPP_W_POINT ? 0.0 : (2.0 * p->nu) * p->eps_R);
  kp.self_pref64 = -(p->dt / p->rho_f) / pow(2.0 * kPi * kp.self_s2, 1.5);
  kp.self_pref = (float)kp.self_pref64;
  kp.raw_norm1 = 1.0 / sqrt(2.0 * kPi * sig2);
  kp.basset_c = p->dt > 0.0 ? 12.0 * (p->rho_f * p->nu) * sqrt(kPi / (p->nu * p->dt)) : 0.0;
  kp.self_inv_w = (float)(1.0 / sqrt(2.0 * kp.self_s2));
  kp.drag_f = (float)(6.0 * kPi * kp.mu);
  kp.rho_f_f = (float)p->rho_f;
  kp.dt_f = (float)p->dt;
  for (int a = 0; a < 3; ++a) {
    kp.grav_f[a] = (float)p->gravity[a];
    kp.halfL_f[a] = (float)(0.5 * L[a]);
    // a position at least 1e-4 L inside the box needs no periodic wrap
    const double wlo = 1e-4 * L[a], whi = (1.0 - 1e-4) * L[a];
    memcpy(&kp.wrap_lo_bits[a], &wlo, sizeof(double));
    memcpy(&kp.wrap_hi_bits[a], &whi, sizeof(double));
  }
  const double log2e = 1.4426950408889634;
  for (int a = 0; a < 3; ++a) {
    kp.beta[a] = (float)(log2e * kp.dx[a] * kp.dx[a] / (2.0 * sig2));
    kp.lap_k[a] = (float)(kp.dx[a] * kp.dx[a] / (sig2 * sig2));
  }
  kp.inv_rho_dV = (float)(1.0 / (p->rho_f * kp.dV));
  kp.normalize = (p->flags & ERPP_NORMALIZE) ? 1 : 0;
  kp.self_removal = (p->flags & ERPP_SELF_REMOVAL) ? 1 : 0;
  kp.kahan = (p->flags & ERPP_KAHAN) ? 1 : 0;
  // Tiles: x-tiles of 64 nodes (a smaller even split for short axes), staged
  // in rows of 96 floats with an x-halo of xhlo nodes below and xhhi above
  // (the whole x-window of every particle whose home cell is in the tile);
  // 8 x 8 in y and z.
  kp.xhlo = (int)floor(kp.cp[0]);
  kp.xhhi = kp.xhlo + 1;
  kp.xlmin = (int)floor(2.0 * kp.cp[0]);
  kp.xxs = (int)floor(2.0 * kp.cp[0] + 1e-6) + 1;
  if (!(p->flags & ERPP_FP64) && kp.xxs > 16) return ERPP_EINVAL;  // FP32: x-windows <= 16
  kp.px = 96;
  const int wmax = std::min(64, kp.px - kp.xhlo - kp.xhhi);
  const int hmax = std::max(kp.xhlo, kp.xhhi);
  kp.T[0] = std::min(wmax, n[0]);
  kp.nt[0] = (n[0] + kp.T[0] - 1) / kp.T[0];
  if (kp.nt[0] > 1 && n[0] - (kp.nt[0] - 1) * kp.T[0] < hmax) {
    // a sliver would be left over: split the axis evenly instead
    kp.T[0] = (n[0] + kp.nt[0] - 1) / kp.nt[0];
    kp.nt[0] = (n[0] + kp.T[0] - 1) / kp.T[0];
  }
  const int wlast = n[0] - (kp.nt[0] - 1) * kp.T[0];
  if (kp.nt[0] > 1 && wlast < hmax) return ERPP_EINVAL;
  const int Tyz[3] = {0, 8, 8};
  int64_t ntiles = kp.nt[0];
  for (int a = 1; a < 3; ++a) {
    kp.T[a] = std::min(Tyz[a], n[a]);
    kp.nt[a] = (n[a] + kp.T[a] - 1) / kp.T[a];
    ntiles *= kp.nt[a];
  }
  if (ntiles > (1 << 24)) return ERPP_EINVAL;
  kp.ntiles = (int)ntiles;
  kp.pxy = kp.px * kp.T[1];
  kp.plane = kp.pxy * kp.T[2];
  if ((size_t)kp.plane * 6 * sizeof(float) > 227 * 1024) return ERPP_EINVAL;

  kp.design = 3;
  kp.halo_per_tile = (int64_t)3 * kp.T[2] * kp.T[1] * (kp.xhlo + kp.xhhi);
  c->maxseg[0] = 1;  // a particle belongs to the x-tile of its home cell
  for (int a = 1; a < 3; ++a) c->maxseg[a] = max_pieces(n[a], kp.T[a], kp.hlo, kp.xs);

  // Design 4 (FP32, windows of at most 16 nodes in x and y): tiles of
  // W x 16 x 4 nodes with x- and y-halos, rows and planes 16 (mod 32) floats
  // apart (see erpp_tiles4.cu); pieces are cut in z only.
  const int yxs = (int)floor(2.0 * kp.cp[1] + 1e-6) + 1;
  if (prec == ERPP_FP32 && kp.xxs <= 16 && yxs <= 16) {
    erpp_kparams k4 = kp;
    k4.design = 4;
    k4.yhlo = (int)floor(kp.cp[1]);
    k4.yhhi = k4.yhlo + 1;
    const int hx = k4.xhlo + k4.xhhi, hy = k4.yhlo + k4.yhhi;
    // Tile widths: the requested size (x: 64), raised to the halo depth so
    // that halo strips reach only the neighbouring tiles; a last (ragged) tile
    // thinner than that becomes an even split, else the tiles grow.
    auto split = [&](int want, int n_axis, int depth, int* T, int* nt) {
      int t = std::min(std::max(want, depth), n_axis);
      int m = (n_axis + t - 1) / t;
      if (m > 1 && n_axis - (m - 1) * t < depth) {
        t = (n_axis + m - 1) / m;
        m = (n_axis + t - 1) / t;
      }
      while (m > 1 && n_axis - (m - 1) * t < depth) {
        ++t;
        m = (n_axis + t - 1) / t;
      }
      *T = t;
      *nt = m;
    };
    const int ymax = std::max(k4.yhlo, k4.yhhi);
    split(64, n[0], hmax, &k4.T[0], &k4.nt[0]);
    split(c->tile_req[0] > 0 ? c->tile_req[0] : 16, n[1], ymax, &k4.T[1], &k4.nt[1]);
    const bool ok_x = k4.nt[0] == 1 || n[0] - (k4.nt[0] - 1) * k4.T[0] >= hmax;
    const bool ok_y = k4.nt[1] == 1 || n[1] - (k4.nt[1] - 1) * k4.T[1] >= ymax;
    k4.nthreads = c->tile_req[2] == 512 ? 512 : 256;
    k4.xoff = (k4.xhlo + 3) & ~3;
    const int need = k4.xoff + k4.T[0] + k4.xhhi;
    k4.px = ((need + 15) / 32) * 32 + 16;  // >= xoff + W + xhhi, 16 (mod 32)
    if (k4.px - 32 >= need) k4.px -= 32;
    k4.pxy = k4.px * (k4.T[1] + hy);
    if (k4.pxy % 32 != 16) k4.pxy += 16;
    // z: 4 planes, fewer when the staged tile would not fit
    const int copies = (p->flags & ERPP_KAHAN) ? 6 : 3;
    auto smem = [&](int tz) {
      erpp_kparams t = k4;
      t.plane = t.pxy * tz;
      return std::max(erpp::smem_bytes4(t, copies, false), erpp::smem_bytes4(t, 3, true)) +
             1024;  // + static shared memory
    };
    int tz = c->tile_req[1] > 0 ? c->tile_req[1] : 4;
    while (tz > 1 && smem(tz) > 227 * 1024) tz >>= 1;
    k4.T[2] = std::min(tz, n[2]);
    k4.nt[2] = (n[2] + k4.T[2] - 1) / k4.T[2];
    k4.plane = k4.pxy * k4.T[2];
    const int64_t nt4 = (int64_t)k4.nt[0] * k4.nt[1] * k4.nt[2];
    const bool fits = smem(k4.T[2]) <= 227 * 1024;
    if (ok_x && ok_y && fits && nt4 <= (1 << 24) && k4.px <= 128 && k4.T[1] + hy <= 64) {
      k4.ntiles = (int)nt4;
      // x-strips, then y-strips from a 16-byte boundary; whole blocks of 4
      k4.ystrip_off = ((int64_t)3 * k4.T[2] * (k4.T[1] + hy) * hx + 3) & ~(int64_t)3;
      k4.halo_per_tile = (k4.ystrip_off + (int64_t)3 * k4.T[2] * hy * k4.T[0] + 3) & ~(int64_t)3;
      kp = k4;
      // x: one piece per window, or two with the windows cut at x-tile
      // boundaries (room for both, so that the scatter mode can change)
      kp.xclip = c->scatter_mode == ERPP_SCATTER_XCLIP ? 1 : 0;
      c->maxseg[0] = max_pieces(n[0], kp.T[0], kp.hlo, kp.xs);
      c->maxseg[1] = 1;
      c->maxseg[2] = max_pieces(n[2], kp.T[2], kp.hlo, kp.xs);
    }
  }

  c->params = *p;
  c->kp = kp;
  c->fp64 = prec == ERPP_FP64;
  c->xw_len = erpp::xw_len(kp);
  return ERPP_OK;
}

}  // namespace erpp

extern "C" {

erpp_status erpp_init(const erpp_params* p, erpp_ctx** out) {
  if (!out) return ERPP_EINVAL;
  *out = nullptr;
  if (!p) return ERPP_EINVAL;
  erpp_ctx* c = (erpp_ctx*)calloc(1, sizeof(erpp_ctx));
  if (!c) return ERPP_ENOMEM;
  erpp_status s0 = erpp::derive_ctx(p, c);
  if (s0 != ERPP_OK) {
    free(c);
    return s0;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->red, sizeof(double) * (6 * 304 + 8));
  c->lag_n = -1;  // the delayed source and the general force start with a first step
  c->ff_n = -1;
  erpp_status st = set_cuda_err(e);
  if (st == ERPP_OK) st = alloc_tile_tables(c);
  if (st == ERPP_OK) st = alloc_weight_tables(c);
  if (st != ERPP_OK) {
    erpp_destroy(c);
    cudaGetLastError();
    return st;
  }
  *out = c;
  return ERPP_OK;
}

erpp_status erpp_destroy(erpp_ctx* c) {
  if (!c) return ERPP_OK;
  cudaDeviceSynchronize();
  erpp::free_host_pipe(c);
  if (c->prof_ev) {
    for (int k = 0; k < kProfSets * 5; ++k) cudaEventDestroy(c->prof_ev[k]);
    free(c->prof_ev);
  }
  free_scratch(c);
  free_tile_tables(c);
  cudaFree(c->w_cnt);
  cudaFree(c->w_start);
  cudaFree(c->w_tmp);
  cudaFree(c->err);
  cudaFree(c->red);
  free(c);
  return ERPP_OK;
}

erpp_status erpp_set_tiling(erpp_ctx* c, int32_t tile_y, int32_t tile_z, int32_t threads) {
  if (!c) return ERPP_EINVAL;
  if (tile_y < 0 || tile_y > 32 || !(tile_z == 0 || tile_z == 1 || tile_z == 2 || tile_z == 4) ||
      !(threads == 0 || threads == 256 || threads == 512))
    return ERPP_EINVAL;
  erpp_ctx probe = *c;
  probe.tile_req[0] = tile_y;
  probe.tile_req[1] = tile_z;
  probe.tile_req[2] = threads;
  erpp_status s = erpp::derive_ctx(&c->params, &probe);
  if (s != ERPP_OK) return s;
  // new geometry: tile tables, halo and piece records are reallocated
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_cuda_err(e);
  free_scratch(c);
  free_tile_tables(c);
  c->tile_req[0] = tile_y;
  c->tile_req[1] = tile_z;
  c->tile_req[2] = threads;
  c->lag_n = -1;  // the delayed source's history went with the scratch: first_step next
  c->ff_n = -1;
  c->kp = probe.kp;
  c->cluster_probe = 0;
  for (int a = 0; a < 3; ++a) c->maxseg[a] = probe.maxseg[a];
  c->xw_len = probe.xw_len;
  return alloc_tile_tables(c);
}

erpp_status erpp_set_scatter_mode(erpp_ctx* c, int32_t mode) {
  if (!c || (mode != ERPP_SCATTER_MERGE && mode != ERPP_SCATTER_CLUSTER &&
             mode != ERPP_SCATTER_XCLIP))
    return ERPP_EINVAL;
  c->scatter_mode = mode;
  c->kp.xclip = (c->kp.design == 4 && mode == ERPP_SCATTER_XCLIP) ? 1 : 0;
  return ERPP_OK;
}

erpp_status erpp_get_tiling(erpp_ctx* c, int32_t out[5]) {
  if (!c || !out) return ERPP_EINVAL;
  out[0] = c->kp.design;
  out[1] = c->kp.T[0];
  out[2] = c->kp.T[1];
  out[3] = c->kp.T[2];
  out[4] = c->kp.design == 4 ? c->kp.nthreads : 256;
  return ERPP_OK;
}

erpp_status erpp_interpolate(erpp_ctx* c, const void* u, int64_t n, const double* const x[3],
                             double* const up[3], erpp_stream stream) {
  if (!c || !u || check_n(n)) return ERPP_EINVAL;
  if (n == 0) return ERPP_OK;
  if (!valid_vec(x) || !up || !up[0] || !up[1] || !up[2]) return ERPP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  erpp_status s = erpp::ensure_capacity(c, n);
  if (s) return s;
  cudaError_t e;
  if (c->kp.weights != ERPP_W_GAUSS) {
    e = erpp::sort_by_cell_block(c, n, x, st);
    if (e == cudaSuccess) e = erpp::launch_gather_weights(c, u, n, x, up, st);
  } else if (c->fp64) {
    e = erpp::launch_gather_f64(c, (const double*)u, n, x, up, st);
  } else {
    e = erpp::bin_particles(c, n, x, true, st);
    if (e == cudaSuccess) e = erpp::launch_gather_f32(c, (const float*)u, n, st);
    if (e == cudaSuccess) e = erpp::launch_finalize_up(c, n, x, up, st);
  }
  return set_cuda_err(e);
}

erpp_status erpp_particle_advance(erpp_ctx* c, const double* const up[3], const erpp_particles* P,
                                  int first_step, erpp_stream stream) {
  if (!c || !P || check_n(P->n)) return ERPP_EINVAL;
  if (P->n == 0) return ERPP_OK;
  if (!up || !up[0] || !up[1] || !up[2] || !P->radius || !P->rho_p) return ERPP_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!P->x[a] || !P->v[a] || !P->x_prev[a] || !P->D[a]) return ERPP_EINVAL;
  cudaError_t e = erpp::launch_advance(c, P, up, false, false, first_step, (cudaStream_t)stream);
  return set_cuda_err(e);
}

erpp_status erpp_scatter_source(erpp_ctx* c, int64_t n, const double* const x[3],
                                const double* const D[3], void* S, erpp_stream stream) {
  if (!c || !S || check_n(n)) return ERPP_EINVAL;
  if (n > 0 && (!valid_vec(x) || !valid_vec(D))) return ERPP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  erpp_status s = erpp::ensure_capacity(c, n);
  if (s) return s;
  return set_cuda_err(erpp::scatter_source(c, n, x, D, S, st));
}

erpp_status erpp_scatter_backward(erpp_ctx* c, int64_t n, const double* const x[3],
                                  const double* const D[3], const void* R, double* const dD[3],
                                  double* const dx[3], erpp_stream stream) {
  if (!c || !R || check_n(n) || c->kp.weights != ERPP_W_GAUSS) return ERPP_EINVAL;
  if (n == 0) return ERPP_OK;
  if (!valid_vec(x) || !valid_vec(D) || !dx || !dx[0] || !dx[1] || !dx[2]) return ERPP_EINVAL;
  if (dD && (!dD[0] || !dD[1] || !dD[2])) return ERPP_EINVAL;
  cudaError_t e = erpp::launch_adjoint(c, n, x, R, D, -1.0 / c->params.rho_f, 0.0, dD, dx,
                                       (cudaStream_t)stream);
  return set_cuda_err(e);
}

erpp_status erpp_gather_backward(erpp_ctx* c, int64_t n, const double* const x[3], const void* u,
                                 const double* const g[3], void* du, double* const dx[3],
                                 erpp_stream stream) {
  if (!c || !u || check_n(n) || c->kp.weights != ERPP_W_GAUSS) return ERPP_EINVAL;
  if (n > 0 && (!valid_vec(x) || !valid_vec(g))) return ERPP_EINVAL;
  if (dx && (!dx[0] || !dx[1] || !dx[2])) return ERPP_EINVAL;
  if (!du && !dx) return ERPP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (dx && n > 0)
    e = erpp::launch_adjoint(c, n, x, u, g, c->kp.dV, c->params.shear_rate, nullptr, dx, st);
  if (e == cudaSuccess && du) {
    erpp_status s = erpp::ensure_capacity(c, n);
    if (s) return s;
    if (c->fp64) {
      e = erpp::launch_scatter_f64(c, n, x, g, c->kp.dV, (double*)du, st);
    } else {
      e = erpp::bin_particles(c, n, x, false, st);
      if (e == cudaSuccess) e = erpp::launch_prep_fscat(c, n, g, 1.0f, st);
      if (e == cudaSuccess) e = erpp::launch_scatter_f32(c, (float*)du, st);
    }
  }
  return set_cuda_err(e);
}

erpp_status erpp_step(erpp_ctx* c, const void* u, const erpp_particles* P, void* S,
                      int first_step, erpp_stream stream) {
  if (!c || !u || !P || !S || check_n(P->n)) return ERPP_EINVAL;
  if (P->n > 0) {
    if (!P->radius || !P->rho_p) return ERPP_EINVAL;
    for (int a = 0; a < 3; ++a)
      if (!P->x[a] || !P->v[a] || !P->x_prev[a] || !P->D[a]) return ERPP_EINVAL;
  }
  return erpp::step_device(c, u, P, S, first_step, (cudaStream_t)stream, nullptr);
}

}  // extern "C"

namespace erpp {

cudaError_t scatter_source(erpp_ctx* c, int64_t n, const double* const x[3],
                           const double* const D[3], void* S, cudaStream_t st) {
  if (c->kp.weights == ERPP_W_PIC) {
    cudaError_t e = erpp::sort_by_cell_block(c, n, x, st);
    if (e != cudaSuccess) return e;
    return erpp::launch_scatter_pic(c, n, x, D, -1.0 / c->params.rho_f, S, st);
  }
  if (c->fp64)
    return erpp::launch_scatter_f64(c, n, x, D, -1.0 / c->params.rho_f, (double*)S, st);
  cudaError_t e = erpp::bin_particles(c, n, x, false, st);
  if (e == cudaSuccess) e = erpp::launch_prep_fscat(c, n, D, -c->kp.inv_rho_dV, st);
  if (e == cudaSuccess) e = erpp::launch_scatter_f32(c, (float*)S, st);
  return e;
}

// The step with the source delayed by L = kp.lag steps (ERPP_LAG): ring slot
// k mod (L + 1) holds (x^k, D^k).  At step n the advance removes the
// disturbance of the source of step n - 1 (slot n - 1 - L), the source is
// slot n - L (none while n < L), and (x^n, D^n) then go to slot n, the one the
// removal has just read.
erpp_status step_lagged(erpp_ctx* c, const void* u, const erpp_particles* P, void* S,
                        int first_step, cudaStream_t st, cudaEvent_t after_advance) {
  const int64_t n = P->n;
  const int64_t L = c->kp.lag;
  if (first_step) {
    c->lag_step = 0;
    c->lag_n = n;
  } else if (n != c->lag_n) {
    return ERPP_ESTATE;
  }
  const int64_t k = c->lag_step;
  const size_t slot_len = (size_t)6 * (size_t)c->cap;
  auto slot = [&](int64_t j) { return c->lag_ring + (size_t)(j % (L + 1)) * slot_len; };
  auto xs_of = [&](double* b, const double* out[3]) {
    for (int a = 0; a < 3; ++a) out[a] = b + (size_t)a * c->cap;
  };
  auto Ds_of = [&](double* b, const double* out[3]) {
    for (int a = 0; a < 3; ++a) out[a] = b + (size_t)(3 + a) * c->cap;
  };
  const double* const xin[3] = {P->x[0], P->x[1], P->x[2]};
  const double* const xprev[3] = {P->x_prev[0], P->x_prev[1], P->x_prev[2]};
  const double* const Dv[3] = {P->D[0], P->D[1], P->D[2]};
  const bool remove = k >= L + 1;
  const double* xs[3] = {nullptr, nullptr, nullptr};
  const double* Ds[3] = {nullptr, nullptr, nullptr};
  if (remove) {
    xs_of(slot(k - 1 - L), xs);
    Ds_of(slot(k - 1 - L), Ds);
  }
  const int no_removal = remove ? 0 : 1;
  cudaError_t e;
  c->launches = 0;
  if (c->fp64) {
    double* up[3] = {c->up64, c->up64 + c->cap, c->up64 + 2 * c->cap};
    e = erpp::launch_gather_f64(c, (const double*)u, n, xin, up, st);
    const double* const upc[3] = {up[0], up[1], up[2]};
    if (e == cudaSuccess)
      e = erpp::launch_advance(c, P, upc, false, false, no_removal, st, remove ? xs : nullptr,
                               remove ? Ds : nullptr);
  } else {
    e = erpp::bin_particles(c, n, xin, true, st);
    if (e == cudaSuccess) e = erpp::launch_gather_f32(c, (const float*)u, n, st);
    if (e == cudaSuccess)
      e = erpp::launch_advance(c, P, nullptr, true, false, no_removal, st, remove ? xs : nullptr,
                               remove ? Ds : nullptr);
  }
  if (e == cudaSuccess && after_advance) e = cudaEventRecord(after_advance, st);
  if (e == cudaSuccess) {
    if (k >= L) {
      const double* xl[3];
      const double* Dl[3];
      xs_of(slot(k - L), xl);
      Ds_of(slot(k - L), Dl);
      e = erpp::scatter_source(c, n, xl, Dl, S, st);
    } else {
      const size_t nn = (size_t)c->kp.n[0] * c->kp.n[1] * c->kp.n[2];
      e = cudaMemsetAsync(S, 0, 3 * nn * (c->fp64 ? sizeof(double) : sizeof(float)), st);
    }
  }
  if (e == cudaSuccess) e = erpp::launch_lag_store(c, n, xprev, Dv, slot(k), st);
  if (e == cudaSuccess) c->lag_step = k + 1;
  c->last_step_launches = c->launches;
  return set_cuda_err(e);
}

// The step with the general force (ERPP_FULL_FORCE): gather of the velocity and
// its Laplacian, the general-force advance, the source of D^n at x^n.  FP32 on
// x/y-halo tiles: one binning of x^n serves the tile gather of both and the
// source (the advance leaves x^n in x_prev); otherwise the warp-per-particle
// gather, and the source binned on its own.
erpp_status step_full_force(erpp_ctx* c, const void* u, const erpp_particles* P, void* S,
                            int first_step, cudaStream_t st, cudaEvent_t after_advance) {
  const int64_t n = P->n;
  if (first_step)
    c->ff_n = n;
  else if (n != c->ff_n)
    return ERPP_ESTATE;
  const double* const xin[3] = {P->x[0], P->x[1], P->x[2]};
  const double* const xprev[3] = {P->x_prev[0], P->x_prev[1], P->x_prev[2]};
  const double* const Dv[3] = {P->D[0], P->D[1], P->D[2]};
  double* up[3] = {c->up64, c->up64 + c->cap, c->up64 + 2 * c->cap};
  const double* const upc[3] = {up[0], up[1], up[2]};
  c->launches = 0;
  const bool tiles = !c->fp64 && c->kp.design == 4 && c->kp.weights == ERPP_W_GAUSS;
  cudaError_t e = cudaSuccess;
  if (tiles) {
    e = erpp::bin_particles(c, n, xin, true, st);
    if (e == cudaSuccess) e = erpp::launch_gather_lap_f32_4(c, (const float*)u, st);
    if (e == cudaSuccess) e = erpp::launch_finalize_full(c, n, xin, up, c->ff_lap, c->cap, st);
  } else {
    e = erpp::launch_gather_faxen(c, u, n, xin, up, st);
  }
  if (e == cudaSuccess) e = erpp::launch_advance_full(c, P, upc, first_step, st);
  if (e == cudaSuccess && after_advance) e = cudaEventRecord(after_advance, st);
  if (e == cudaSuccess && tiles) {
    e = erpp::launch_prep_fscat(c, n, Dv, -c->kp.inv_rho_dV, st);
    if (e == cudaSuccess) e = erpp::launch_scatter_f32(c, (float*)S, st);
  } else if (e == cudaSuccess) {
    e = erpp::scatter_source(c, n, xprev, Dv, S, st);
  }
  c->last_step_launches = c->launches;
  return set_cuda_err(e);
}

erpp_status step_device(erpp_ctx* c, const void* u, const erpp_particles* P, void* S,
                        int first_step, cudaStream_t st, cudaEvent_t after_advance) {
  const int64_t n = P->n;
  erpp_status s = erpp::ensure_capacity(c, n);
  if (s) return s;
  if (c->kp.lag > 0) return step_lagged(c, u, P, S, first_step, st, after_advance);
  if (c->kp.full_force) return step_full_force(c, u, P, S, first_step, st, after_advance);
  const double* const xin[3] = {P->x[0], P->x[1], P->x[2]};
  const double* const xprev[3] = {P->x_prev[0], P->x_prev[1], P->x_prev[2]};
  const double* const Dv[3] = {P->D[0], P->D[1], P->D[2]};
  cudaError_t e;
  c->launches = 0;
  if (c->kp.weights != ERPP_W_GAUSS) {
    // other weights: gather into up64, advance from it, scatter D^n at x^n
    // (the PIC source reuses the order of the gather: x_prev holds x^n after
    // the advance)
    double* up[3] = {c->up64, c->up64 + c->cap, c->up64 + 2 * c->cap};
    e = erpp::sort_by_cell_block(c, n, xin, st);
    if (e == cudaSuccess) e = erpp::launch_gather_weights(c, u, n, xin, up, st);
    const double* const upc[3] = {up[0], up[1], up[2]};
    if (e == cudaSuccess) e = erpp::launch_advance(c, P, upc, false, false, first_step, st);
    if (e == cudaSuccess && after_advance) e = cudaEventRecord(after_advance, st);
    if (e == cudaSuccess) {
      if (c->kp.weights == ERPP_W_PIC)
        e = erpp::launch_scatter_pic(c, n, xprev, Dv, -1.0 / c->params.rho_f, S, st);
      else
        e = erpp::scatter_source(c, n, xprev, Dv, S, st);
    }
  } else if (c->fp64) {
    double* up[3] = {c->up64, c->up64 + c->cap, c->up64 + 2 * c->cap};
    e = erpp::launch_gather_f64(c, (const double*)u, n, xin, up, st);
    const double* const upc[3] = {up[0], up[1], up[2]};
    if (e == cudaSuccess) e = erpp::launch_advance(c, P, upc, false, false, first_step, st);
    if (e == cudaSuccess && after_advance) e = cudaEventRecord(after_advance, st);
    if (e == cudaSuccess)
      e = erpp::launch_scatter_f64(c, n, xprev, Dv, -1.0 / c->params.rho_f, (double*)S, st);
  } else {
    cudaEvent_t* ev = nullptr;
    if (c->prof_on) ev = c->prof_ev + 5 * (c->prof_n++ % kProfSets);
    if (ev) cudaEventRecord(ev[0], st);
    e = erpp::bin_particles(c, n, xin, true, st);
    if (ev) cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = erpp::launch_gather_f32(c, (const float*)u, n, st);
    if (ev) cudaEventRecord(ev[2], st);
    if (e == cudaSuccess) e = erpp::launch_advance(c, P, nullptr, true, true, first_step, st);
    if (e == cudaSuccess && after_advance) e = cudaEventRecord(after_advance, st);
    if (ev) cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = erpp::launch_scatter_f32(c, (float*)S, st);
    if (ev) cudaEventRecord(ev[4], st);
  }
  c->last_step_launches = c->launches;
  return set_cuda_err(e);
}

}  // namespace erpp

extern "C" {

erpp_status erpp_last_step_launches(erpp_ctx* c, int32_t* n) {
  if (!c || !n) return ERPP_EINVAL;
  *n = c->last_step_launches;
  return ERPP_OK;
}

erpp_status erpp_profile_enable(erpp_ctx* c, int enable) {
  if (!c) return ERPP_EINVAL;
  if (enable && !c->prof_ev) {
    c->prof_ev = (cudaEvent_t*)calloc((size_t)kProfSets * 5, sizeof(cudaEvent_t));
    if (!c->prof_ev) return ERPP_ENOMEM;
    for (int k = 0; k < kProfSets * 5; ++k) {
      cudaError_t e = cudaEventCreate(&c->prof_ev[k]);
      if (e != cudaSuccess) return set_cuda_err(e);
    }
  }
  c->prof_on = enable ? 1 : 0;
  return ERPP_OK;
}

erpp_status erpp_profile_read(erpp_ctx* c, double ms[4], int64_t* steps) {
  if (!c || !ms || !steps) return ERPP_EINVAL;
  for (int k = 0; k < 4; ++k) ms[k] = 0.0;
  *steps = 0;
  if (!c->prof_ev) return ERPP_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_cuda_err(e);
  int nsets = c->prof_n < kProfSets ? c->prof_n : kProfSets;
  for (int s = 0; s < nsets; ++s) {
    cudaEvent_t* ev = c->prof_ev + 5 * s;
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      if (e != cudaSuccess) return set_cuda_err(e);
      ms[k] += t;
    }
  }
  *steps = nsets;
  c->prof_n = 0;
  return ERPP_OK;
}

erpp_status erpp_check(erpp_ctx* c, erpp_stream stream) {
  if (!c) return ERPP_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return set_cuda_err(e);
  uint32_t h = 0;
  e = cudaMemcpy(&h, c->err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_cuda_err(e);
  if (h) {
    e = cudaMemset(c->err, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return set_cuda_err(e);
  }
  if (h & ERPP_ERRBIT_RANGE) return ERPP_ERANGE;
  if (h & ERPP_ERRBIT_BOUNDS) return ERPP_EBOUNDS;
  if (h & ERPP_ERRBIT_TIMEOUT) return ERPP_ETIMEOUT;
  return ERPP_OK;
}

erpp_status erpp_momentum(erpp_ctx* c, const void* S, int64_t n, const double* const x[3],
                          const double* const D[3], double out[6], erpp_stream stream) {
  if (!c || !S || !out || check_n(n)) return ERPP_EINVAL;
  if (n > 0 && (!valid_vec(x) || !valid_vec(D))) return ERPP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = erpp::launch_momentum(c, S, n, x, D, st);
  if (e != cudaSuccess) return set_cuda_err(e);
  e = cudaMemcpyAsync(out, c->red + 6 * 304, sizeof(double) * 6, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return set_cuda_err(e);
  return erpp_check(c, stream);
}

erpp_status erpp_debug_set_wait(erpp_ctx* c, int64_t limit_ns, int32_t stall) {
  if (!c || limit_ns < 0 || limit_ns > 10000000000LL || (stall != 0 && stall != 1))
    return ERPP_EINVAL;
  if (limit_ns > 0 && limit_ns < 1000) return ERPP_EINVAL;
  c->wait_req_ns = limit_ns;
  c->stall_req = stall;
  c->kp.wait_ns = limit_ns > 0 ? limit_ns : kDefaultWaitNs;
  c->kp.debug_stall = stall;
  return ERPP_OK;
}

erpp_status erpp_debug_windows(erpp_ctx* c, int64_t n, const double* const x[3], int32_t* jlo,
                               int32_t* jhi, erpp_stream stream) {
  if (!c || check_n(n)) return ERPP_EINVAL;
  if (n == 0) return ERPP_OK;
  if (!valid_vec(x) || !jlo || !jhi) return ERPP_EINVAL;
  return set_cuda_err(erpp::launch_windows(c, n, x, jlo, jhi, (cudaStream_t)stream));
}

}  // extern "C"
