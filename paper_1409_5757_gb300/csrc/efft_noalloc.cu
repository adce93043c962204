// efft_noalloc.cu -- efft_execute_noalloc: one transform with no allocation.
//
// Some callers cannot call cudaMalloc: a framework whose pooled allocator
// owns all device memory, or a pipeline that cannot afford cudaMalloc's
// implicit device-wide synchronisation.  For them this entry point runs the
// same kernels as efft_execute with the plan's twiddle tables and state word
// placed in the file-scope device array below instead of in plan-owned
// allocations.  The caller passes only the data buffer.
//
// The array is a device symbol: in host code its name is only a stand-in, so
// the host obtains its device address with cudaGetSymbolAddress (once per
// device, on the first call with that device current) and hands that
// address to the kernels.  Every GPU that loads the library holds the array
// until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/efft.h"

// Implemented in efft.cu: runs one transform with tables and state in
// `scratch` (device memory of `scratch_bytes`), regenerating the twiddle
// tables first when `regen` is set.
int efft_internal_run_in_scratch(void* scratch, size_t scratch_bytes, bool regen, void* data, uint64_t n,
                                 int dtype, int sign, uint32_t flags, cudaStream_t st);

namespace {

// twiddle tables for N <= 2^24: 2048 + 2^12 + 2^12 float4, then 16 bytes of state
constexpr size_t kScratchBytes = (2048 + 4096 + 4096) * 16 + 256;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_tables_log2n[kMaxDevices];
bool g_init_done = false;

}  // namespace

extern "C" int efft_execute_noalloc(void* data, uint64_t n, int dtype, int sign, uint32_t flags, void* stream) {
  if (n == 0 || (n & (n - 1)) != 0 || n > (1ull << EFFT_NOALLOC_MAX_LOG2N)) return EFFT_ERR_INVALID_SIZE;
  if (dtype != EFFT_C64 && dtype != EFFT_C128) return EFFT_ERR_INVALID_DTYPE;
  if (sign != -1 && sign != 1) return EFFT_ERR_INVALID_SIGN;
  if (flags & ~(EFFT_FLAG_DIGIT_REVERSED_OUT | EFFT_FLAG_NORMALIZE)) return EFFT_ERR_INVALID_FLAGS;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return EFFT_ERR_UNSUPPORTED;
  int log2n = 0;
  while ((1ull << log2n) < n) ++log2n;

  void* base = nullptr;
  bool regen = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_init_done) {
      for (int i = 0; i < kMaxDevices; ++i) g_tables_log2n[i] = -1;
      g_init_done = true;
    }
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t err = cudaGetSymbolAddress(&ptr, g_scratch);
      if (err != cudaSuccess || !ptr) {
        cudaGetLastError();
        return EFFT_ERR_CUDA;
      }
      g_addr[dev] = ptr;
    }
    base = g_addr[dev];
    regen = (g_tables_log2n[dev] != log2n);
    // The tables are enqueued on this call's stream; a later call with the same
    // N reuses them (calls that overlap on the GPU race, as documented).
    if (regen) g_tables_log2n[dev] = log2n;
  }
  int rc = efft_internal_run_in_scratch(base, kScratchBytes, regen, data, n, dtype, sign, flags,
                                        reinterpret_cast<cudaStream_t>(stream));
  if (rc != EFFT_OK && regen) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tables_log2n[dev] = -1;  // tables may be incomplete: rebuild next time
  }
  return rc;
}
