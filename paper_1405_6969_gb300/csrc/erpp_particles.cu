// erpp_particles.cu -- per-particle kernels: self-disturbance removal, Stokes
// drag and explicit Euler advance (Sec. 2.5), the general-force advance of
// Eq. force_particle, normalisation of the gathered velocity, the scatter's
// force words, the delayed source's ring store, momentum sums and debug
// windows.
#include <cuda_runtime.h>

#include "erpp_internal.cuh"

namespace {

struct PartPtrs {
  double* x[3];
  double* v[3];
  double* xp[3];
  double* D[3];
  const double* radius;
  const double* rho_p;
  // position and force of the source whose disturbance is removed: x_prev and
  // D (the previous step's) unless the source is delayed by eps_R
  const double* xs[3];
  const double* Ds[3];
};

struct UpPtrs {
  const double* up[3];
};

__device__ __forceinline__ double min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
  if (x < 0.0) x = x + L;
  if (x >= L) x = x - L;
  return x;
}

// Closed-form regularised disturbance of App. A.5 (Eq. disturbance_velo),
// prefactor -dt/rho_f included, variance self_s2:
//   v = pref { [e^-eta^2 - F(eta)] D - (D.rh) [e^-eta^2 - 3 F(eta)] rh },
//   F(eta) = f(eta) / (2 eta^3), f(eta) = (sqrt(pi)/2) erf(eta) - eta e^-eta^2.
// Below eta = 1/2 the two terms of f cancel; there F is summed from its
// Taylor series sum_k (-1)^k eta^2k / (k! (2k+3)).
__device__ void self_velocity_f32(const erpp_kparams& kp, const float r[3], const float D[3],
                                  float out[3]) {
  float rr = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  float eta = rr * kp.self_inv_w;
  float e2 = eta * eta;
  float e = expf(-e2);
  float F;
  if (eta < 0.5f) {
    float term = 1.f, sum = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sum += term / (float)(2 * k + 3);
      term = -term * e2 / (float)(k + 1);
    }
    F = sum;
  } else {
    float f = 0.886226925452758f * erff(eta) - eta * e;
    F = f / (2.f * eta * e2);
  }
  float rh[3] = {0.f, 0.f, 0.f};
  float Ddr = 0.f;
  if (rr > 0.f) {
    float inv = 1.f / rr;
    rh[0] = r[0] * inv;
    rh[1] = r[1] * inv;
    rh[2] = r[2] * inv;
    Ddr = D[0] * rh[0] + D[1] * rh[1] + D[2] * rh[2];
  }
  float c1 = e - F, c2 = Ddr * (e - 3.f * F);
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = kp.self_pref * (c1 * D[a] - c2 * rh[a]);
}

__device__ void self_velocity_f64(const erpp_kparams& kp, const double r[3], const double D[3],
                                  double out[3]) {
  const double pi = 3.141592653589793238462643;
  double s2 = kp.self_s2;
  double pref = kp.self_pref64;
  double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  double eta = rr / sqrt(2.0 * s2);
  double F;
  if (eta < 0.5) {
    double e2 = eta * eta, term = 1.0, sum = 0.0;
    for (int k = 0; k < 20; ++k) {
      sum += term / (double)(2 * k + 3);
      term = -term * e2 / (double)(k + 1);
    }
    F = sum;
  } else {
    double f = 0.5 * sqrt(pi) * erf(eta) - eta * exp(-eta * eta);
    F = f / (2.0 * eta * eta * eta);
  }
  double e = exp(-eta * eta);
  double rh[3] = {0.0, 0.0, 0.0};
  double Ddr = 0.0;
  if (rr > 0.0) {
    for (int a = 0; a < 3; ++a) rh[a] = r[a] / rr;
    Ddr = D[0] * rh[0] + D[1] * rh[1] + D[2] * rh[2];
  }
  for (int a = 0; a < 3; ++a) out[a] = pref * ((e - F) * D[a] - Ddr * (e - 3.0 * F) * rh[a]);
}

// Laplacian in r of the disturbance above: the disturbance is the Leray
// projection of a Gaussian of variance s2, and d g/d s2 = (1/2) lap g, so
// lap v = 2 dv/ds2 at fixed dt/rho_f.  With v = pref(s2) B(eta),
// pref ~ s2^(-3/2), eta = r / sqrt(2 s2):  lap v = -(pref / s2)(3 B + eta dB/deta),
// dB/deta = [e' - F'] D - (D.rh)[e' - 3 F'] rh, e' = -2 eta e^-eta^2,
// F' = e^-eta^2 / eta - 3 F / eta (series below eta = 1/2).
__device__ void self_laplacian_f64(const erpp_kparams& kp, const double r[3], const double D[3],
                                   double out[3]) {
  const double pi = 3.141592653589793238462643;
  const double s2 = kp.self_s2;
  const double pref = kp.self_pref64;
  const double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const double eta = rr / sqrt(2.0 * s2);
  const double e = exp(-eta * eta);
  double F, dF;
  if (eta < 0.5) {
    double e2 = eta * eta, term = 1.0, sum = 0.0, dsum = 0.0;
    for (int k = 0; k < 20; ++k) {
      sum += term / (double)(2 * k + 3);
      dsum += (double)(2 * k) * term / (double)(2 * k + 3);
      term = -term * e2 / (double)(k + 1);
    }
    F = sum;
    dF = eta > 0.0 ? dsum / eta : 0.0;
  } else {
    const double f = 0.5 * sqrt(pi) * erf(eta) - eta * e;
    F = f / (2.0 * eta * eta * eta);
    dF = e / eta - 3.0 * F / eta;
  }
  const double de = -2.0 * eta * e;
  double rh[3] = {0.0, 0.0, 0.0};
  double Ddr = 0.0;
  if (rr > 0.0) {
    for (int a = 0; a < 3; ++a) rh[a] = r[a] / rr;
    Ddr = D[0] * rh[0] + D[1] * rh[1] + D[2] * rh[2];
  }
  for (int a = 0; a < 3; ++a) {
    const double B = (e - F) * D[a] - Ddr * (e - 3.0 * F) * rh[a];
    const double dB = (de - dF) * D[a] - Ddr * (de - 3.0 * dF) * rh[a];
    out[a] = -(pref / s2) * (3.0 * B + eta * dB);
  }
}

// The same in FP32 (the closed forms of the FP32 step): series below eta = 1/2.
__device__ void self_laplacian_f32(const erpp_kparams& kp, const float r[3], const float D[3],
                                   float out[3]) {
  const float rr = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  const float eta = rr * kp.self_inv_w;
  const float e = expf(-eta * eta);
  float F, dF;
  if (eta < 0.5f) {
    float e2 = eta * eta, term = 1.f, sum = 0.f, dsum = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sum += term / (float)(2 * k + 3);
      dsum += (float)(2 * k) * term / (float)(2 * k + 3);
      term = -term * e2 / (float)(k + 1);
    }
    F = sum;
    dF = eta > 0.f ? dsum / eta : 0.f;
  } else {
    const float f = 0.886226925452758f * erff(eta) - eta * e;
    F = f / (2.f * eta * eta * eta);
    dF = e / eta - 3.f * F / eta;
  }
  const float de = -2.f * eta * e;
  float rh[3] = {0.f, 0.f, 0.f};
  float Ddr = 0.f;
  if (rr > 0.f) {
    const float inv = 1.f / rr;
    for (int a = 0; a < 3; ++a) rh[a] = r[a] * inv;
    Ddr = D[0] * rh[0] + D[1] * rh[1] + D[2] * rh[2];
  }
  const float c = -kp.self_pref / (float)kp.self_s2;
  for (int a = 0; a < 3; ++a) {
    const float B = (e - F) * D[a] - Ddr * (e - 3.f * F) * rh[a];
    const float dB = (de - dF) * D[a] - Ddr * (de - 3.f * dF) * rh[a];
    out[a] = c * (3.f * B + eta * dB);
  }
}

// The general force of Eq. force_particle (ERPP_FULL_FORCE), one thread per
// particle in FP64: self removal of the velocity and of its Laplacian, Faxen
// slip q - v (q = u~ + (a^2/6) lap u~), fluid-acceleration and added-mass
// terms from the change of u~ over the last step (prev: u~ and lap u~ of the
// previous step, [6][stride]; none on a first step), one-step Basset memory
// c_B (q - q_prev), the particle's own added mass and memory at the step's
// velocity change, Euler update.
// F32: the closed forms of the removed disturbance in FP32 (as in the FP32
// Stokes-drag step); the force terms and the update in FP64.
template <bool F32>
__global__ void __launch_bounds__(256) k_advance_full(erpp_kparams kp, int64_t n, PartPtrs P,
                                                      UpPtrs U, const double* __restrict__ lap,
                                                      double* __restrict__ prev, int64_t stride,
                                                      int first_step) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double pi = 3.141592653589793238462643;
  double x[3], v[3], ut[3], Lt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = P.x[a][i];
    v[a] = P.v[a][i];
    ut[a] = U.up[a][i];
    Lt[a] = lap[a * stride + i];
  }
  if (kp.self_removal && !first_step) {
    double r[3], D[3], vs[3], ls[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      r[a] = min_image(x[a] - P.xp[a][i], kp.L[a]);
      D[a] = P.D[a][i];
    }
    if (F32) {
      const float rf[3] = {(float)r[0], (float)r[1], (float)r[2]};
      const float Df[3] = {(float)D[0], (float)D[1], (float)D[2]};
      float vf[3], lf[3];
      self_velocity_f32(kp, rf, Df, vf);
      self_laplacian_f32(kp, rf, Df, lf);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        vs[a] = (double)vf[a];
        ls[a] = (double)lf[a];
      }
    } else {
      self_velocity_f64(kp, r, D, vs);
      self_laplacian_f64(kp, r, D, ls);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ut[a] -= vs[a];
      Lt[a] -= ls[a];
    }
  }
  double up_prev[3], Lp_prev[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    up_prev[a] = first_step ? ut[a] : prev[a * stride + i];
    Lp_prev[a] = first_step ? Lt[a] : prev[(3 + a) * stride + i];
  }
  const double a_p = P.radius[i];
  const double a2 = a_p * a_p;
  const double vol = (4.0 / 3.0) * pi * a_p * a2;
  const double m_p = vol * P.rho_p[i];
  const double m_f = vol * kp.rho_f;
  const double dt = kp.dt;
  const double c_B = kp.basset_c * a2;
  const double k_drag = 6.0 * pi * kp.mu * a_p;
  // one division per particle: the FP64 divide is slow on this part
  const double mf_dt = m_f / dt;
  const double inv_M = 1.0 / (m_p / dt + 0.5 * mf_dt + c_B);
  const double c_D = 0.5 * mf_dt + c_B;
  const double a2_6 = a2 * (1.0 / 6.0), a2_10 = a2 * 0.1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double q = ut[a] + a2_6 * Lt[a];
    const double q_prev = up_prev[a] + a2_6 * Lp_prev[a];
    const double F = k_drag * (q - v[a]) + mf_dt * (ut[a] - up_prev[a]) +
                     0.5 * mf_dt * ((ut[a] + a2_10 * Lt[a]) - (up_prev[a] + a2_10 * Lp_prev[a])) +
                     c_B * (q - q_prev);
    const double dv = (F + (m_p - m_f) * kp.gravity[a]) * inv_M;
    P.D[a][i] = F - c_D * dv;
    P.v[a][i] = v[a] + dv;
    P.x[a][i] = wrap_coord(x[a] + dt * v[a], kp.L[a]);
    P.xp[a][i] = x[a];
    prev[a * stride + i] = ut[a];
    prev[(3 + a) * stride + i] = Lt[a];
  }
}

// Removal + drag + Euler (Sec. 2.5, Eqs. particle_motion, force_stokes_drag).
// FROM_ACC: the gathered velocity comes from the tile gather's accumulator
// (scaled here by the kernel normalisation); otherwise from caller arrays.
// F32: the drag and the velocity increment are formed in FP32 from the FP64
// slip (the increment is a small correction to the FP64 velocity); the
// velocity and position updates themselves stay in FP64.
template <bool FROM_ACC, bool F32>
__device__ __forceinline__ void advance_one(const erpp_kparams& kp, int64_t i, const PartPtrs& P,
                                            const UpPtrs& U, const erpp_acc& acc,
                                            const float4* __restrict__ geo_t,
                                            const int4* __restrict__ geo_c,
                                            float4* __restrict__ fscat, int first_step) {
  double x[3], v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = P.x[a][i];
    v[a] = P.v[a][i];
  }
  // F32: the gathered velocity and the self term are FP32 quantities; they
  // are combined in FP32 and the particle velocity is subtracted in FP64.
  double up[3];
  float upf[3] = {0.f, 0.f, 0.f};
  float norm = 0.f;
  if (FROM_ACC) {
    const float4 gt = geo_t[i];
    norm = erpp_norm(kp, gt, geo_c[i]);
    erpp_gathered(kp, acc, gt, i, upf);
#pragma unroll
    for (int a = 0; a < 3; ++a) upf[a] *= norm;
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) up[a] = U.up[a][i];
  }
  double vs[3] = {0.0, 0.0, 0.0};
  float vsf[3] = {0.f, 0.f, 0.f};
  if (kp.self_removal && !first_step) {
    double r[3], D[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double d = x[a] - P.xs[a][i];
      // the exact minimum-image test only where the float difference is
      // near half the box
      r[a] = fabsf(erpp_d2f(d)) > 0.99f * kp.halfL_f[a] ? min_image(d, kp.L[a]) : d;
      D[a] = P.Ds[a][i];
    }
    if (F32) {
      // conversions by integer operations (erpp_d2f): same values, off the
      // FP64 pipe that bounds this kernel
      float rf[3] = {erpp_d2f(r[0]), erpp_d2f(r[1]), erpp_d2f(r[2])};
      float Df[3] = {erpp_d2f(D[0]), erpp_d2f(D[1]), erpp_d2f(D[2])};
      self_velocity_f32(kp, rf, Df, vsf);
    } else {
      self_velocity_f64(kp, r, D, vs);
    }
  }
  const double pi = 3.141592653589793238462643;
  const double a_p = P.radius[i];
  const double rho = P.rho_p[i];
  double Dn[3];
  float Dnf[3];
  if (F32) {
    const float af = erpp_d2f(a_p), rf = erpp_d2f(rho);
    const float k_drag = kp.drag_f * af;
    const float inv_m = 1.f / ((float)(4.0 / 3.0 * pi) * af * af * af * rf);
    const float buoy = 1.f - kp.rho_f_f / rf;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // tile gather: FP32 velocity, plus the mean shear at the particle;
      // caller's FP64 velocity (shear included): subtract in FP64
      double ut;
      if (FROM_ACC) {
        ut = erpp_f2d(upf[a] - vsf[a]);
        if (a == 0) ut += kp.shear_rate * x[1];
      } else {
        ut = up[a] - erpp_f2d(vsf[a]);
      }
      const float slip = erpp_d2f(ut - v[a]);
      const float Df = k_drag * slip;
      const float dv = kp.dt_f * (Df * inv_m + buoy * kp.grav_f[a]);
      Dnf[a] = Df;
      Dn[a] = erpp_f2d(Df);
      P.v[a][i] = v[a] + erpp_f2d(dv);
      double xn = x[a] + kp.dt * v[a];
      // inside [1e-4 L, (1 - 1e-4) L] no wrap is needed (an integer compare
      // of the bit patterns; negative values and NaN fall outside)
      const int64_t xb = __double_as_longlong(xn);
      if (!(xb > kp.wrap_lo_bits[a] && xb < kp.wrap_hi_bits[a])) xn = wrap_coord(xn, kp.L[a]);
      P.x[a][i] = xn;
      P.xp[a][i] = x[a];
      P.D[a][i] = Dn[a];
    }
  } else {
    const double k_drag = 6.0 * pi * kp.mu * a_p;
    const double m_p = (4.0 / 3.0) * pi * a_p * a_p * a_p * rho;
    const double buoy = 1.0 - kp.rho_f / rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Dnf[a] = 0.f;
      double ut = up[a] - vs[a];
      Dn[a] = k_drag * (ut - v[a]);
      P.v[a][i] = v[a] + kp.dt * (Dn[a] / m_p + buoy * kp.gravity[a]);
      P.x[a][i] = wrap_coord(x[a] + kp.dt * v[a], kp.L[a]);
      P.xp[a][i] = x[a];
      P.D[a][i] = Dn[a];
    }
  }
  if (fscat) {
    const float s = -norm * kp.inv_rho_dV;
    const float f0 = s * Dnf[0], f1 = s * Dnf[1], f2 = s * Dnf[2];
    fscat[i] = make_float4(f0, f1, f2, fmaxf(fabsf(f0), fmaxf(fabsf(f1), fabsf(f2))));
  }
}

// The FP32 tile step's advance is bound by its memory traffic: six blocks
// per SM (40 registers, a few spilled) keep more loads in flight, measured
// faster than four (54 registers).
template <bool FROM_ACC, bool F32>
__global__ void __launch_bounds__(256, FROM_ACC && F32 ? 6 : 1)
    k_advance(erpp_kparams kp, int64_t n, PartPtrs P, UpPtrs U, erpp_acc acc,
              const float4* __restrict__ geo_t, const int4* __restrict__ geo_c,
              float4* __restrict__ fscat, int first_step) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  advance_one<FROM_ACC, F32>(kp, i, P, U, acc, geo_t, geo_c, fscat, first_step);
}

// Many boxes in one launch (batched boxes): one block per (box, first
// particle) item of 256 particles; the FP32 tile step's advance of each.
__global__ void __launch_bounds__(256) k_advance_multi(const erpp_box_dev* __restrict__ boxes,
                                                       const int2* __restrict__ items,
                                                       int first_step) {
  const int2 it = items[blockIdx.x];
  const erpp_box_dev& B = boxes[it.x];
  const int64_t i = (int64_t)it.y + threadIdx.x;
  if (i >= B.n) return;
  PartPtrs P;
  for (int a = 0; a < 3; ++a) {
    P.x[a] = B.x[a];
    P.v[a] = B.v[a];
    P.xp[a] = B.xp[a];
    P.D[a] = B.D[a];
    P.xs[a] = B.xp[a];
    P.Ds[a] = B.D[a];
  }
  P.radius = B.radius;
  P.rho_p = B.rho_p;
  UpPtrs U = {{nullptr, nullptr, nullptr}};
  erpp_acc acc;
  acc.up_acc = nullptr;
  acc.stride = B.cap;
  acc.up_part = B.up_part;
  acc.piece_slot = B.piece_slot;
  acc.n = B.n;
  advance_one<true, true>(B.kp, i, P, U, acc, B.geo_t, B.geo_c, B.fscat, first_step);
}

__global__ void k_finalize_up(erpp_kparams kp, int64_t n, erpp_acc acc,
                              const float4* __restrict__ geo_t, const int4* __restrict__ geo_c,
                              const double* __restrict__ y, double* up0, double* up1,
                              double* up2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 gt = geo_t[i];
  const float norm = erpp_norm(kp, gt, geo_c[i]);
  float g[3];
  erpp_gathered(kp, acc, gt, i, g);
  up0[i] = (double)(g[0] * norm) + kp.shear_rate * y[i];
  up1[i] = (double)(g[1] * norm);
  up2[i] = (double)(g[2] * norm);
}

// The general force on x/y-halo tiles: the gathered velocity (norm * sum +
// shear y in x) and its Laplacian (norm * sum of the second-derivative
// weights), each particle's pieces added in piece order.
__global__ void k_finalize_full(erpp_kparams kp, int64_t n, erpp_acc acc,
                                const float4* __restrict__ lap_part,
                                const float4* __restrict__ geo_t, const int4* __restrict__ geo_c,
                                const double* __restrict__ y, double* up0, double* up1,
                                double* up2, double* __restrict__ lap, int64_t lap_stride) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 gt = geo_t[i];
  const float norm = erpp_norm(kp, gt, geo_c[i]);
  float g[3];
  erpp_gathered(kp, acc, gt, i, g);
  const int np = __float_as_int(gt.w);
  float l0 = 0.f, l1 = 0.f, l2 = 0.f;
  for (int k = 0; k < np; ++k) {
    const float4 v = lap_part[acc.piece_slot[(int64_t)k * acc.n + i]];
    l0 += v.x;
    l1 += v.y;
    l2 += v.z;
  }
  up0[i] = (double)(g[0] * norm) + kp.shear_rate * y[i];
  up1[i] = (double)(g[1] * norm);
  up2[i] = (double)(g[2] * norm);
  lap[i] = (double)(l0 * norm);
  lap[lap_stride + i] = (double)(l1 * norm);
  lap[2 * lap_stride + i] = (double)(l2 * norm);
}

erpp_acc acc_of(const erpp_ctx* ctx, int64_t n) {
  erpp_acc a;
  a.up_acc = ctx->up_acc;
  a.stride = ctx->cap;
  a.up_part = ctx->up_part;
  a.piece_slot = ctx->piece_slot;
  a.n = n;
  return a;
}

__global__ void k_prep_fscat(erpp_kparams kp, int64_t n, const double* __restrict__ D0,
                             const double* __restrict__ D1, const double* __restrict__ D2,
                             const float4* __restrict__ geo_t, const int4* __restrict__ geo_c,
                             float scale, float4* __restrict__ fscat) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = erpp_norm(kp, geo_t[i], geo_c[i]) * scale;
  const float f0 = s * (float)D0[i], f1 = s * (float)D1[i], f2 = s * (float)D2[i];
  fscat[i] = make_float4(f0, f1, f2, fmaxf(fabsf(f0), fmaxf(fabsf(f1), fabsf(f2))));
}

__global__ void k_windows(erpp_kparams kp, int64_t n, const double* __restrict__ x0,
                          const double* __restrict__ x1, const double* __restrict__ x2,
                          int32_t* jlo, int32_t* jhi) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* xs[3] = {x0, x1, x2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // the binning's window, checked against the FP64 form: INT32_MIN marks
    // a position where any of its values (home cell, ends, fractional
    // position) differs
    double s, lo, hi;
    erpp_axis_window(xs[a][i], kp.inv_dx[a], kp.cp[a], &s, &lo, &hi);
    const erpp_axis_win aw =
        erpp_axis_window_lean(xs[a][i], kp.inv_dx[a], kp.cp[a], kp.cp_int[a], kp.cp_frac[a]);
    const int ci = (int)floor(s);
    const float t = (float)(s - floor(s));
    const bool same = aw.ci == ci && aw.lo == (int)lo && aw.hi == (int)hi && aw.t == t;
    jlo[a * n + i] = same ? aw.lo : INT32_MIN;
    jhi[a * n + i] = same ? aw.hi : INT32_MIN;
  }
}

// ---------------------------------------------------------------- momentum
constexpr int kRedBlocks = 304;

template <typename T>
__global__ void k_grid_sum(const T* __restrict__ S, size_t nn, double* __restrict__ part) {
  __shared__ double sh[3][8];
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < nn;
       j += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += (double)S[c * nn + j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    part[threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
}

__device__ double axis_mass(const erpp_kparams& kp, int a, double x) {
  double s, lo, hi;
  erpp_axis_window(x, kp.inv_dx[a], kp.cp[a], &s, &lo, &hi);
  const double raw1 = 1.0 / sqrt(2.0 * 3.141592653589793238462643 * kp.sig2);
  double sum = 0.0;
  for (double j = lo; j <= hi; j += 1.0) {
    double d = (j - s) * kp.dx[a];
    sum += raw1 * exp(-(d * d) / (2.0 * kp.sig2));
  }
  return kp.dx[a] * sum;
}

__global__ void k_part_sum(erpp_kparams kp, int64_t n, const double* __restrict__ x0,
                           const double* __restrict__ x1, const double* __restrict__ x2,
                           const double* __restrict__ D0, const double* __restrict__ D1,
                           const double* __restrict__ D2, double* __restrict__ part) {
  __shared__ double sh[3][8];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double M = 1.0;  // trilinear (PIC) weights always carry unit mass
    if (!kp.normalize && kp.weights != ERPP_W_PIC)
      M = axis_mass(kp, 0, x0[i]) * axis_mass(kp, 1, x1[i]) * axis_mass(kp, 2, x2[i]);
    acc[0] += M * D0[i];
    acc[1] += M * D1[i];
    acc[2] += M * D2[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    part[threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
}

// out[0..2] = dV * grid sums, out[3..5] = -(1/rho_f) * particle sums
__global__ void k_momentum_final(erpp_kparams kp, const double* __restrict__ gpart,
                                 const double* __restrict__ ppart, int nb, double* out) {
  int c = threadIdx.x;
  if (c >= 6) return;
  const double* src = c < 3 ? gpart + c * nb : ppart + (c - 3) * nb;
  double v = 0.0;
  for (int k = 0; k < nb; ++k) v += src[k];
  out[c] = c < 3 ? kp.dV * v : -v / kp.rho_f;
}

}  // namespace

namespace erpp {

static PartPtrs part_ptrs(const erpp_particles* P) {
  PartPtrs q;
  for (int a = 0; a < 3; ++a) {
    q.x[a] = P->x[a];
    q.v[a] = P->v[a];
    q.xp[a] = P->x_prev[a];
    q.D[a] = P->D[a];
    q.xs[a] = P->x_prev[a];
    q.Ds[a] = P->D[a];
  }
  q.radius = P->radius;
  q.rho_p = P->rho_p;
  return q;
}

cudaError_t launch_advance(erpp_ctx* ctx, const erpp_particles* P, const double* const up[3],
                           bool from_acc, bool write_fscat, int first_step, cudaStream_t st,
                           const double* const xs[3], const double* const Ds[3]) {
  const int64_t n = P->n;
  if (n <= 0) return cudaSuccess;
  PartPtrs q = part_ptrs(P);
  if (xs && Ds)
    for (int a = 0; a < 3; ++a) {
      q.xs[a] = xs[a];
      q.Ds[a] = Ds[a];
    }
  UpPtrs U;
  for (int a = 0; a < 3; ++a) U.up[a] = up ? up[a] : nullptr;
  int blocks = (int)((n + 255) / 256);
  float4* fs = write_fscat ? ctx->fscat : nullptr;
  const bool f32 = !ctx->fp64;
  ++ctx->launches;
  if (from_acc) {
    k_advance<true, true><<<blocks, 256, 0, st>>>(ctx->kp, n, q, U, acc_of(ctx, n), ctx->geo_t,
                                                  ctx->geo_c, fs, first_step);
  } else if (f32) {
    k_advance<false, true><<<blocks, 256, 0, st>>>(ctx->kp, n, q, U, erpp_acc{}, nullptr,
                                                   nullptr, nullptr, first_step);
  } else {
    k_advance<false, false><<<blocks, 256, 0, st>>>(ctx->kp, n, q, U, erpp_acc{}, nullptr,
                                                    nullptr, nullptr, first_step);
  }
  return cudaGetLastError();
}

cudaError_t launch_advance_full(erpp_ctx* ctx, const erpp_particles* P,
                                const double* const up[3], int first_step, cudaStream_t st) {
  const int64_t n = P->n;
  if (n <= 0) return cudaSuccess;
  PartPtrs q = part_ptrs(P);
  UpPtrs U;
  for (int a = 0; a < 3; ++a) U.up[a] = up[a];
  ++ctx->launches;
  const int blocks = (int)((n + 255) / 256);
  if (ctx->fp64)
    k_advance_full<false><<<blocks, 256, 0, st>>>(ctx->kp, n, q, U, ctx->ff_lap, ctx->ff_prev,
                                                  ctx->cap, first_step);
  else
    k_advance_full<true><<<blocks, 256, 0, st>>>(ctx->kp, n, q, U, ctx->ff_lap, ctx->ff_prev,
                                                 ctx->cap, first_step);
  return cudaGetLastError();
}

// ring[slot] <- (x^n, D^n): six arrays of n doubles, [x0 x1 x2 D0 D1 D2].
__global__ void k_lag_store(int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
                            const double* __restrict__ x2, const double* __restrict__ D0,
                            const double* __restrict__ D1, const double* __restrict__ D2,
                            double* __restrict__ slot, int64_t stride) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    slot[i] = x0[i];
    slot[stride + i] = x1[i];
    slot[2 * stride + i] = x2[i];
    slot[3 * stride + i] = D0[i];
    slot[4 * stride + i] = D1[i];
    slot[5 * stride + i] = D2[i];
  }
}

cudaError_t launch_lag_store(erpp_ctx* ctx, int64_t n, const double* const x[3],
                             const double* const D[3], double* slot, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  ++ctx->launches;
  k_lag_store<<<(int)b, 256, 0, st>>>(n, x[0], x[1], x[2], D[0], D[1], D[2], slot, ctx->cap);
  return cudaGetLastError();
}

cudaError_t launch_finalize_up(erpp_ctx* ctx, int64_t n, const double* const x[3],
                               double* const up[3], cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  ++ctx->launches;
  k_finalize_up<<<blocks, 256, 0, st>>>(ctx->kp, n, acc_of(ctx, n), ctx->geo_t, ctx->geo_c,
                                        x[1], up[0], up[1], up[2]);
  return cudaGetLastError();
}

cudaError_t launch_finalize_full(erpp_ctx* ctx, int64_t n, const double* const x[3],
                                 double* const up[3], double* lap, int64_t lap_stride,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  ++ctx->launches;
  k_finalize_full<<<blocks, 256, 0, st>>>(ctx->kp, n, acc_of(ctx, n), ctx->lap_part, ctx->geo_t,
                                          ctx->geo_c, x[1], up[0], up[1], up[2], lap, lap_stride);
  return cudaGetLastError();
}

cudaError_t launch_prep_fscat(erpp_ctx* ctx, int64_t n, const double* const D[3], float scale,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  ++ctx->launches;
  k_prep_fscat<<<blocks, 256, 0, st>>>(ctx->kp, n, D[0], D[1], D[2], ctx->geo_t, ctx->geo_c,
                                       scale, ctx->fscat);
  return cudaGetLastError();
}

cudaError_t launch_windows(erpp_ctx* ctx, int64_t n, const double* const x[3], int32_t* jlo,
                           int32_t* jhi, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  k_windows<<<blocks, 256, 0, st>>>(ctx->kp, n, x[0], x[1], x[2], jlo, jhi);
  return cudaGetLastError();
}

cudaError_t launch_momentum(erpp_ctx* ctx, const void* S, int64_t n, const double* const x[3],
                            const double* const D[3], cudaStream_t st) {
  const erpp_kparams& kp = ctx->kp;
  size_t nn = (size_t)kp.n[0] * kp.n[1] * kp.n[2];
  double* gpart = ctx->red;
  double* ppart = ctx->red + 3 * kRedBlocks;
  double* out = ctx->red + 6 * kRedBlocks;
  if (ctx->fp64)
    k_grid_sum<double><<<kRedBlocks, 256, 0, st>>>((const double*)S, nn, gpart);
  else
    k_grid_sum<float><<<kRedBlocks, 256, 0, st>>>((const float*)S, nn, gpart);
  k_part_sum<<<kRedBlocks, 256, 0, st>>>(kp, n, x[0], x[1], x[2], D[0], D[1], D[2], ppart);
  k_momentum_final<<<1, 32, 0, st>>>(kp, gpart, ppart, kRedBlocks, out);
  return cudaGetLastError();
}


cudaError_t launch_advance_multi(const erpp_box_dev* boxes, const int2* pitems, int npitems,
                                 int first_step, cudaStream_t st) {
  if (npitems > 0) k_advance_multi<<<npitems, 256, 0, st>>>(boxes, pitems, first_step);
  return cudaGetLastError();
}

}  // namespace erpp
