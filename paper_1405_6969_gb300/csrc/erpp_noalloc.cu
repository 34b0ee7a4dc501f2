// erpp_noalloc.cu -- an interpolation entry point that allocates nothing.
//
// erpp_interpolate needs a context, and creating one (erpp_init) allocates
// device memory.  Some callers cannot allocate: code that runs while a memory
// pool is frozen or exhausted, plugins that receive a fixed device budget from
// their host application, or paths that must not call into the allocator at
// all.  erpp_interpolate_noalloc serves them for small problems: it runs the
// same FP32 tile gather with its scratch (particle geometry, stencil pieces,
// per-tile tables) carved out of one fixed array in device memory that is
// part of the library image, so no cudaMalloc, cudaFree or other allocating
// call is ever made.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "erpp_internal.cuh"

namespace {

constexpr int64_t kNoallocParticles = 16384;       // particles per call, at most
constexpr int64_t kNoallocPieces = 8 * kNoallocParticles;
constexpr int64_t kNoallocTiles = 4096;            // grid tiles, at most

// Byte layout of the static scratch (each part 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffGeoT = 0;
constexpr size_t kOffGeoC = kOffGeoT + align256(16 * kNoallocParticles);
constexpr size_t kOffAcc = kOffGeoC + align256(16 * kNoallocParticles);
constexpr size_t kOffXw = kOffAcc + align256(12 * kNoallocParticles);
constexpr size_t kOffEntries = kOffXw + align256(4 * 16 * kNoallocParticles);
constexpr int64_t kNoallocBins = 32 * kNoallocTiles;  // (tile, bucket) bins
constexpr size_t kOffCnt = kOffEntries + align256(16 * kNoallocPieces);
constexpr size_t kOffStart = kOffCnt + align256(4 * kNoallocBins);
constexpr size_t kOffSlot = kOffStart + align256(4 * (kNoallocBins + 1));
constexpr size_t kOffScan = kOffSlot + align256(4 * kNoallocPieces);
constexpr size_t kOffPart = kOffScan + align256(4 * (kNoallocBins / 4096 + 1));
constexpr size_t kOffErr = kOffPart + align256(16 * kNoallocPieces);
constexpr size_t kScratchBytes = kOffErr + 256;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];
static_assert(kScratchBytes < 10u * 1024u * 1024u, "no-alloc scratch must stay modest");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the unique id of the CUDA context the address was looked up in,
// and the address.  A context created later on the same device (after a
// reset, or another context) has another id and its own copy of the array.
unsigned long long g_ctx_id[kMaxDevices] = {0};
unsigned char* g_dev_addr[kMaxDevices] = {nullptr};

typedef int (*ctx_get_current_fn)(void**);
typedef int (*ctx_get_id_fn)(void*, unsigned long long*);

// Unique id of the calling thread's current CUDA context (driver entry points
// through the runtime, no link against the driver library); 0 when unknown.
unsigned long long current_ctx_id() {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<ctx_get_current_fn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<ctx_get_id_fn>(p);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch in the current context, looked up (with the
// device current) the first time each context calls; without a context id
// the address is looked up on every call.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (id == 0 || g_ctx_id[dev] != id || !g_dev_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_addr[dev] = (unsigned char*)p;
    g_ctx_id[dev] = id;
  }
  *out = g_dev_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" erpp_status erpp_interpolate_noalloc(const erpp_params* params, const void* u,
                                                int64_t n, const double* const x[3],
                                                double* const u_p[3], erpp_stream stream) {
  if (!params || !u) return ERPP_EINVAL;
  if ((params->flags & (ERPP_FP32 | ERPP_FP64)) != ERPP_FP32) return ERPP_EINVAL;
  if (params->flags & (ERPP_PIC | ERPP_POINT_GATHER)) return ERPP_EINVAL;
  if (n < 0 || n > kNoallocParticles) return ERPP_EINVAL;
  if (n > 0 && (!x || !x[0] || !x[1] || !x[2] || !u_p || !u_p[0] || !u_p[1] || !u_p[2]))
    return ERPP_EINVAL;
  erpp_ctx c;
  memset(&c, 0, sizeof(c));
  erpp_status s = erpp::derive_ctx(params, &c);
  if (s != ERPP_OK) return s;
  const int64_t pieces = n * (int64_t)c.maxseg[0] * c.maxseg[1] * c.maxseg[2];
  if (c.kp.ntiles > kNoallocTiles || pieces > kNoallocPieces) return ERPP_EINVAL;
  if (n == 0) return ERPP_OK;
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return ERPP_ECUDA;
  c.cap = kNoallocParticles;
  c.entries_cap = kNoallocPieces;
  c.geo_t = reinterpret_cast<float4*>(base + kOffGeoT);
  c.geo_c = reinterpret_cast<int4*>(base + kOffGeoC);
  c.up_acc = reinterpret_cast<float*>(base + kOffAcc);
  c.entries = reinterpret_cast<int4*>(base + kOffEntries);
  c.xw = reinterpret_cast<float*>(base + kOffXw);
  // the x/y-halo tiles keep one x-distance per particle where the x-halo
  // tiles keep their x-weights (a context uses one of the two)
  c.d0x = reinterpret_cast<float*>(base + kOffXw);
  c.tile_cnt = reinterpret_cast<int32_t*>(base + kOffCnt);
  c.tile_start = reinterpret_cast<int32_t*>(base + kOffStart);
  c.piece_slot = reinterpret_cast<int32_t*>(base + kOffSlot);
  c.scan_tmp = reinterpret_cast<int32_t*>(base + kOffScan);
  c.up_part = reinterpret_cast<float4*>(base + kOffPart);
  c.err = reinterpret_cast<uint32_t*>(base + kOffErr);
  cudaStream_t st = (cudaStream_t)stream;
  // The per-tile counts are cleared by the binning itself and the gather
  // accumulators by its first pass; the error word is cleared here.
  e = cudaMemsetAsync(c.err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = erpp::bin_particles(&c, n, x, true, st);
  if (e == cudaSuccess) e = erpp::launch_gather_f32(&c, (const float*)u, n, st);
  if (e == cudaSuccess) e = erpp::launch_finalize_up(&c, n, x, u_p, st);
  return e == cudaSuccess ? ERPP_OK : ERPP_ECUDA;
}
