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
// context, on the first call with that context current) and hands that
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
namespace efft {
namespace host {
int current_context(int* dev, unsigned long long* ctx_id);
}  // namespace host
}  // namespace efft

namespace {

// twiddle tables for N <= 2^24: 2048 + 2^12 + 2^12 float4, then 16 bytes of state
constexpr size_t kScratchBytes = (2048 + 4096 + 4096) * 16 + 256;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// What the host knows about the array in one context: its device address
// and the log2 N whose tables it holds (-1: none, or not known to be
// complete).  A context is identified by its device and the driver's
// context ID, so a context created after a device reset starts afresh.
struct Known {
  int dev;
  unsigned long long ctx;
  void* addr;
  int tables_log2n;
};
constexpr int kMaxContexts = 64;
std::mutex g_mu;
Known g_known[kMaxContexts];
int g_nknown = 0;

Known* find_or_add(int dev, unsigned long long ctx) {
  for (int i = 0; i < g_nknown; ++i)
    if (g_known[i].dev == dev && g_known[i].ctx == ctx) return &g_known[i];
  if (g_nknown == kMaxContexts) {  // full: drop the oldest context's entry
    for (int i = 1; i < kMaxContexts; ++i) g_known[i - 1] = g_known[i];
    --g_nknown;
  }
  Known* k = &g_known[g_nknown++];
  *k = Known{dev, ctx, nullptr, -1};
  return k;
}

}  // namespace

extern "C" int efft_execute_noalloc(void* data, uint64_t n, int dtype, int sign, uint32_t flags, void* stream) {
  if (n == 0 || (n & (n - 1)) != 0 || n > (1ull << EFFT_NOALLOC_MAX_LOG2N)) return EFFT_ERR_INVALID_SIZE;
  if (dtype != EFFT_C64 && dtype != EFFT_C128) return EFFT_ERR_INVALID_DTYPE;
  if (sign != -1 && sign != 1) return EFFT_ERR_INVALID_SIGN;
  if (flags & ~(EFFT_FLAG_DIGIT_REVERSED_OUT | EFFT_FLAG_NORMALIZE)) return EFFT_ERR_INVALID_FLAGS;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  unsigned long long ctx = 0;
  if (efft::host::current_context(&dev, &ctx) != EFFT_OK) return EFFT_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  if (cs == cudaStreamCaptureStatusInvalidated) return EFFT_ERR_CUDA;
  const bool capturing = (cs == cudaStreamCaptureStatusActive);
  int log2n = 0;
  while ((1ull << log2n) < n) ++log2n;

  void* base = nullptr;
  bool regen = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    Known* k = find_or_add(dev, ctx);
    if (!k->addr) {
      void* ptr = nullptr;
      cudaError_t err = cudaGetSymbolAddress(&ptr, g_scratch);
      if (err != cudaSuccess || !ptr) {
        cudaGetLastError();
        return EFFT_ERR_CUDA;
      }
      k->addr = ptr;
    }
    base = k->addr;
    if (capturing) {
      // A captured call runs when its graph is launched, after any number of
      // other calls: it regenerates its own tables at every launch, and the
      // next eager call rebuilds them too (the graph's launches overwrite
      // whatever the array held).
      regen = true;
      k->tables_log2n = -1;
    } else {
      regen = (k->tables_log2n != log2n);
      // the tables are enqueued on this call's stream; a later call with the
      // same N reuses them (calls that overlap on the GPU race, as documented)
      if (regen) k->tables_log2n = log2n;
    }
  }
  int rc = efft_internal_run_in_scratch(base, kScratchBytes, regen, data, n, dtype, sign, flags, st);
  if (rc != EFFT_OK && regen && !capturing) {
    std::lock_guard<std::mutex> lk(g_mu);
    Known* k = find_or_add(dev, ctx);
    k->tables_log2n = -1;  // tables may be incomplete: rebuild next time
  }
  return rc;
}
