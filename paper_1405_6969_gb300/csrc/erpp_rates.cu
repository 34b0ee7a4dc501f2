// erpp_rates.cu -- the measured rate of the shared-memory atomic add that the
// scatter's accumulation is built on.
//
// In the scatter (Sec. 2.4, Eq. ns_regularized_filtered) every node of every
// particle's truncated stencil receives one contribution per force
// component; the tile kernels add each one to the staged tile with one
// shared-memory atomic add (a 32-bit fixed-point integer, or an FP32 value on
// dense tiles).  This file measures how many such adds the GPU completes per
// second when nothing else limits them: every SM full of warps whose lanes
// add to 32 distinct banks, unrolled so that the loop costs little beside the
// adds.  A measurement aid, not part of the method.
#include <cuda_runtime.h>

#include "../../include/erpp.h"

namespace {

constexpr int kRateThreads = 256;
constexpr int kRateUnroll = 16;   // adds per thread per loop iteration
constexpr int kRateIters = 2048;  // loop iterations per thread

// Adds J.. of one iteration: word a + 32 J of the warp's block of words
// (lane l at bank l).
template <int J, bool F32>
__device__ __forceinline__ void rate_adds(unsigned a) {
  if constexpr (J < kRateUnroll) {
    if constexpr (F32)
      asm volatile("red.shared.add.f32 [%0+%1], %2;\n" ::"r"(a), "n"(128 * J), "f"(1.f));
    else
      asm volatile("red.shared.add.s32 [%0+%1], %2;\n" ::"r"(a), "n"(128 * J), "r"(1));
    rate_adds<J + 1, F32>(a);
  }
}

// Warp w owns words [w 32 kRateUnroll, (w + 1) 32 kRateUnroll) of the block's
// kRateThreads kRateUnroll words; *out receives a flag that keeps the sums
// live.
template <bool F32>
__global__ void __launch_bounds__(kRateThreads) k_shared_add_rate(int iters, int* out) {
  __shared__ int words[kRateThreads * kRateUnroll];
  for (int k = threadIdx.x; k < kRateThreads * kRateUnroll; k += kRateThreads) words[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned a =
      (unsigned)__cvta_generic_to_shared(words + warp * 32 * kRateUnroll + lane);
  for (int it = 0; it < iters; ++it) rate_adds<0, F32>(a);
  __syncthreads();
  if (threadIdx.x == 0 && words[0] != 0) atomicOr(out, 1);
}

erpp_status status_of(cudaError_t e) {
  if (e == cudaSuccess) return ERPP_OK;
  return e == cudaErrorMemoryAllocation ? ERPP_ENOMEM : ERPP_ECUDA;
}

}  // namespace

extern "C" erpp_status erpp_shared_add_rate(int32_t kind, double* adds_per_s) {
  if (!adds_per_s || (kind != ERPP_RATE_SHARED_S32 && kind != ERPP_RATE_SHARED_F32))
    return ERPP_EINVAL;
  *adds_per_s = 0.0;
  auto kern = kind == ERPP_RATE_SHARED_F32 ? k_shared_add_rate<true> : k_shared_add_rate<false>;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRateThreads, 0);
  if (e == cudaSuccess && (nsm < 1 || per_sm < 1)) return ERPP_ECUDA;
  int* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  // one block per resident slot of every SM; the first launch warms up, the
  // fastest of the others is kept
  const int blocks = nsm * per_sm;
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(ev[0], st);
    if (e != cudaSuccess) break;
    kern<<<blocks, kRateThreads, 0, st>>>(kRateIters, out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && rep > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess && best > 0.f)
    *adds_per_s = (double)blocks * kRateThreads * (double)kRateIters * kRateUnroll /
                  ((double)best * 1e-3);
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return status_of(e);
}
