// erpp_fluid.cu -- the fluid stand-in: one exact step of the periodic
// unsteady Stokes equations forced by the regularised source.
//
// The paper couples the particles to a pseudo-spectral DNS (Sec. 3-4); the
// coupling step only needs a fluid that responds to S.  This stand-in
// advances the linear disturbance problem of Sec. 2.2 with the forcing,
// projection and diffusion split that App. A.5 uses for one time step:
//   u_hat <- exp(-nu |k|^2 dt) P(k) (u_hat + dt S_hat),
// P(k) = I - k k^T / |k|^2 the Leray projector (identity on the mean mode),
// wavenumbers k_a = 2 pi m_a / L_a with m_a the signed FFT index (on the
// Nyquist planes of even axes, the mean projector of the mode and its mirror).
// Transforms: cuFFT real-to-complex / complex-to-real over the three
// components (batched); the spectral update (projection, decay and the
// 1/N normalisation of the round trip) is one kernel of this file, one
// thread per complex coefficient.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <stdlib.h>

#include "erpp_internal.cuh"

struct erpp_fluid {
  int32_t n[3];
  double L[3];
  double nu, dt;
  int fp64;
  size_t nspec;     // complex coefficients per component: nz * ny * (nx/2 + 1)
  void* spec;       // [3][nspec] complex (float2 or double2)
  cufftHandle r2c;
  cufftHandle c2r;
  int have_r2c, have_c2r;
};

namespace {

template <typename T>
__global__ void k_add_scaled(T* __restrict__ u, const T* __restrict__ S, T dt, size_t total) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x)
    u[i] += dt * S[i];
}

// Signed frequency of FFT index i on n points (the Nyquist index of an even
// n counts as -n/2), and whether i is that Nyquist index.
__device__ __forceinline__ double signed_index(int i, int n) {
  return (double)(i < (n + 1) / 2 ? i : i - n);
}
__device__ __forceinline__ bool nyquist(int i, int n) { return (n & 1) == 0 && i == n / 2; }

template <typename C, typename T>
__global__ void k_spectral(C* __restrict__ spec, size_t nspec, int nxh, int ny, int nz, int nx,
                           T kx0, T ky0, T kz0, T nu_dt, T inv_n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nspec;
       i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nxh);
    const size_t r = i / nxh;
    const int iy = (int)(r % ny);
    const int iz = (int)(r / ny);
    const T kx = kx0 * (T)signed_index(ix, nx);
    const T ky = ky0 * (T)signed_index(iy, ny);
    const T kz = kz0 * (T)signed_index(iz, nz);
    const T k2 = kx * kx + ky * ky + kz * kz;
    // On a Nyquist plane the mode m and its mirror -m share the frequency of
    // the Nyquist component, so the projector of the real field is the mean
    // of P(k) and P(k~), k~ = k with its Nyquist components negated (what
    // projecting every coefficient of the full transform and keeping the
    // real part gives).  Elsewhere k~ = k.
    const T tx = nyquist(ix, nx) ? -kx : kx;
    const T ty = nyquist(iy, ny) ? -ky : ky;
    const T tz = nyquist(iz, nz) ? -kz : kz;
    C a = spec[i], b = spec[nspec + i], c = spec[2 * nspec + i];
    if (k2 > (T)0) {
      const T inv = (T)0.5 / k2;
      const T pr = (kx * a.x + ky * b.x + kz * c.x) * inv;
      const T pi = (kx * a.y + ky * b.y + kz * c.y) * inv;
      const T qr = (tx * a.x + ty * b.x + tz * c.x) * inv;
      const T qi = (tx * a.y + ty * b.y + tz * c.y) * inv;
      a.x -= kx * pr + tx * qr;
      a.y -= kx * pi + tx * qi;
      b.x -= ky * pr + ty * qr;
      b.y -= ky * pi + ty * qi;
      c.x -= kz * pr + tz * qr;
      c.y -= kz * pi + tz * qi;
    }
    const T f = exp(-nu_dt * k2) * inv_n;
    a.x *= f;
    a.y *= f;
    b.x *= f;
    b.y *= f;
    c.x *= f;
    c.y *= f;
    spec[i] = a;
    spec[nspec + i] = b;
    spec[2 * nspec + i] = c;
  }
}

int grid_blocks(size_t total) {
  size_t b = (total + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

extern "C" {

erpp_status erpp_fluid_destroy(erpp_fluid* f) {
  if (!f) return ERPP_OK;
  cudaDeviceSynchronize();
  if (f->have_r2c) cufftDestroy(f->r2c);
  if (f->have_c2r) cufftDestroy(f->c2r);
  cudaFree(f->spec);
  free(f);
  return ERPP_OK;
}

erpp_status erpp_fluid_init(const erpp_params* p, erpp_fluid** out) {
  if (!out) return ERPP_EINVAL;
  *out = nullptr;
  if (!p) return ERPP_EINVAL;
  const uint32_t prec = p->flags & (ERPP_FP32 | ERPP_FP64);
  if (prec != ERPP_FP32 && prec != ERPP_FP64) return ERPP_EINVAL;
  const int32_t n[3] = {p->nx, p->ny, p->nz};
  const double L[3] = {p->Lx, p->Ly, p->Lz};
  for (int a = 0; a < 3; ++a)
    if (n[a] < 2 || !(L[a] > 0.0) || !isfinite(L[a])) return ERPP_EINVAL;
  if (!(p->nu >= 0.0) || !(p->dt > 0.0) || !isfinite(p->nu) || !isfinite(p->dt))
    return ERPP_EINVAL;
  erpp_fluid* f = (erpp_fluid*)calloc(1, sizeof(erpp_fluid));
  if (!f) return ERPP_ENOMEM;
  for (int a = 0; a < 3; ++a) {
    f->n[a] = n[a];
    f->L[a] = L[a];
  }
  f->nu = p->nu;
  f->dt = p->dt;
  f->fp64 = prec == ERPP_FP64;
  f->nspec = (size_t)n[2] * n[1] * (n[0] / 2 + 1);
  const size_t csz = f->fp64 ? sizeof(double2) : sizeof(float2);
  cudaError_t e = cudaMalloc(&f->spec, 3 * f->nspec * csz);
  if (e != cudaSuccess) {
    erpp_fluid_destroy(f);
    cudaGetLastError();
    return ERPP_ENOMEM;
  }
  int dims[3] = {n[2], n[1], n[0]};
  const long long real_dist = (long long)n[2] * n[1] * n[0];
  int inembed[3] = {n[2], n[1], n[0]};
  int onembed[3] = {n[2], n[1], n[0] / 2 + 1};
  cufftResult r = cufftPlanMany(&f->r2c, 3, dims, inembed, 1, (int)real_dist, onembed, 1,
                                (int)f->nspec, f->fp64 ? CUFFT_D2Z : CUFFT_R2C, 3);
  f->have_r2c = r == CUFFT_SUCCESS;
  if (r == CUFFT_SUCCESS)
    r = cufftPlanMany(&f->c2r, 3, dims, onembed, 1, (int)f->nspec, inembed, 1, (int)real_dist,
                      f->fp64 ? CUFFT_Z2D : CUFFT_C2R, 3);
  f->have_c2r = f->have_r2c && r == CUFFT_SUCCESS;
  if (r != CUFFT_SUCCESS) {
    erpp_fluid_destroy(f);
    cudaGetLastError();
    return r == CUFFT_ALLOC_FAILED ? ERPP_ENOMEM : ERPP_ECUDA;
  }
  *out = f;
  return ERPP_OK;
}

erpp_status erpp_fluid_stokes_step(erpp_fluid* f, void* u, const void* S, erpp_stream stream) {
  if (!f || !u || !S) return ERPP_EINVAL;
  if ((size_t)f->n[0] * f->n[1] * f->n[2] * 3 > (size_t)1 << 40) return ERPP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t total = 3 * (size_t)f->n[0] * f->n[1] * f->n[2];
  const double kx0 = 2.0 * 3.141592653589793238462643 / f->L[0];
  const double ky0 = 2.0 * 3.141592653589793238462643 / f->L[1];
  const double kz0 = 2.0 * 3.141592653589793238462643 / f->L[2];
  const double inv_n = 1.0 / ((double)f->n[0] * f->n[1] * f->n[2]);
  const int nxh = f->n[0] / 2 + 1;
  if (cufftSetStream(f->r2c, st) != CUFFT_SUCCESS || cufftSetStream(f->c2r, st) != CUFFT_SUCCESS)
    return ERPP_ECUDA;
  cufftResult r;
  if (f->fp64) {
    k_add_scaled<double><<<grid_blocks(total), 256, 0, st>>>((double*)u, (const double*)S, f->dt,
                                                             total);
    r = cufftExecD2Z(f->r2c, (cufftDoubleReal*)u, (cufftDoubleComplex*)f->spec);
    if (r == CUFFT_SUCCESS)
      k_spectral<double2, double><<<grid_blocks(f->nspec), 256, 0, st>>>(
          (double2*)f->spec, f->nspec, nxh, f->n[1], f->n[2], f->n[0], kx0, ky0, kz0,
          f->nu * f->dt, inv_n);
    if (r == CUFFT_SUCCESS)
      r = cufftExecZ2D(f->c2r, (cufftDoubleComplex*)f->spec, (cufftDoubleReal*)u);
  } else {
    k_add_scaled<float><<<grid_blocks(total), 256, 0, st>>>((float*)u, (const float*)S,
                                                            (float)f->dt, total);
    r = cufftExecR2C(f->r2c, (cufftReal*)u, (cufftComplex*)f->spec);
    if (r == CUFFT_SUCCESS)
      k_spectral<float2, float><<<grid_blocks(f->nspec), 256, 0, st>>>(
          (float2*)f->spec, f->nspec, nxh, f->n[1], f->n[2], f->n[0], (float)kx0, (float)ky0,
          (float)kz0, (float)(f->nu * f->dt), (float)inv_n);
    if (r == CUFFT_SUCCESS) r = cufftExecC2R(f->c2r, (cufftComplex*)f->spec, (cufftReal*)u);
  }
  if (r != CUFFT_SUCCESS) return ERPP_ECUDA;
  return cudaGetLastError() == cudaSuccess ? ERPP_OK : ERPP_ECUDA;
}

}  // extern "C"
