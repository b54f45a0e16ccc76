// love_noalloc.cu -- K_UU product for callers that cannot allocate device memory.
//
// ski_mvm_kuu needs a work area for the FFT of grid modes longer than 2048
// points (a four-step transform that goes through global memory) and takes it
// from the handle's allocator.  Some callers cannot allocate at that point: a
// real-time loop that forbids allocator calls (an allocation can block on a
// lock or synchronise the device), a host framework that owns and has already
// reserved all device memory, or code running inside the caching allocator's
// own callbacks, which cannot re-enter it.  ski_mvm_kuu_noalloc gives them the
// same product with its scratch in a fixed, file-scope device array.
//
// Scratch: LOVE_NOALLOC_SCRATCH_BYTES (4 MiB) of device memory, present on every
// GPU that loads this library, for the life of the process.  It holds
// N x (m / g_e) complex doubles for the longest mode with g_e > 2048, so a 1-D
// grid of up to 131,072 points (or Kronecker modes of the same product size).
// Larger grids are rejected with LOVE_ERR_UNSUPPORTED.
#include <mutex>

#include "love_internal.cuh"

#define LOVE_NOALLOC_SCRATCH_BYTES (4u << 20)

static __device__ __align__(256) unsigned char g_kuu_scratch[LOVE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_kuu_scratch on the current device (looked up once per device)
love_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return love::cuda_check(e);
  if (dev < 0 || dev >= kMaxDevices) return LOVE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_kuu_scratch);
    if (e != cudaSuccess || !p) return love::cuda_check(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LOVE_OK;
}

}  // namespace

extern "C" LOVE_API love_status ski_mvm_kuu_noalloc(love_ski_t ski, const void* v, void* out,
                                                    love_stream_t stream) try {
  if (!ski || !v || !out) return LOVE_ERR_ARG;
  const GridHost& g = ski->grid;
  const size_t need = love::fft_work_bytes(g, ski->fft, 1, true);
  if (need > LOVE_NOALLOC_SCRATCH_BYTES) return LOVE_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  if (need > 0) LOVE_TRY(scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  if (ski->dtype == LOVE_F64)
    return love::kuu_apply<double>(g, ski->fft, (const double*)v, (double*)out, 1, g.m, scratch, -1, s);
  return love::kuu_apply<float>(g, ski->fft, (const float*)v, (float*)out, 1, g.m, scratch, -1, s);
}
LOVE_ENTRY_CATCH
