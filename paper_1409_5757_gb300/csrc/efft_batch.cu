// efft_batch.cu -- batches of independent in-place transforms of mixed
// power-of-two sizes behind one CUDA graph (efft_batch_* in include/efft.h).
// Transforms of one size share a plan and run in the same launches (grid.y
// selects the transform); the sizes run as parallel branches of the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "../../include/efft.h"
#include "efft_host.h"

using namespace efft;
using namespace efft::host;

struct efft_batch_s {
  uint32_t magic = 0;
  int device = 0;
  int count = 0;
  std::vector<efft_plan_s*> plans;  // one per distinct size, largest first
  std::vector<int> gstart;          // group g owns pointer slots [gstart[g], gstart[g+1])
  std::vector<int> slot;            // transform i -> its pointer slot
  std::vector<int> group;           // transform i -> its group
  void** dptrs = nullptr;           // device: count pointers, by slot
  uint32_t* state = nullptr;        // device: 16 bytes per slot
  void** stage = nullptr;           // pinned host: EFFT_BATCH_INFLIGHT * count pointers
  cudaEvent_t done[EFFT_BATCH_INFLIGHT] = {};
  int next = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

namespace {

constexpr uint32_t kBatchMagic = 0xEFF7BA7Cu;
std::set<efft_batch_s*>* g_live_batches = nullptr;  // leaked on purpose, guarded by registry_mutex()

bool batch_is_live(efft_batch_s* b) {
  std::lock_guard<std::mutex> lk(registry_mutex());
  return g_live_batches && g_live_batches->count(b) && b->magic == kBatchMagic;
}

void batch_free(efft_batch_s* b) {
  for (int k = 0; k < EFFT_BATCH_INFLIGHT; ++k)
    if (b->done[k]) cudaEventSynchronize(b->done[k]);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int k = 0; k < EFFT_BATCH_INFLIGHT; ++k)
    if (b->done[k]) cudaEventDestroy(b->done[k]);
  if (b->dptrs) cudaFree(b->dptrs);
  if (b->state) cudaFree(b->state);
  if (b->stage) cudaFreeHost(b->stage);
  for (efft_plan_s* p : b->plans) efft_plan_destroy(p);
  cudaGetLastError();
  delete b;
}

// Records every group's launches into one graph: group 0 on the capture
// stream, the others on forked side streams joined back at the end.
int batch_capture(efft_batch_s* b) {
  const int G = (int)b->plans.size();
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> side(G, nullptr);
  std::vector<cudaEvent_t> join(G, nullptr);
  cudaEvent_t fork = nullptr;
  int rc = EFFT_OK;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
    rc = EFFT_ERR_CUDA;
  for (int g = 1; rc == EFFT_OK && g < G; ++g)
    if (cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&join[g], cudaEventDisableTiming) != cudaSuccess)
      rc = EFFT_ERR_CUDA;
  if (rc == EFFT_OK) {
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = EFFT_ERR_CUDA;
    } else {
      bool forked = (G == 1) || cudaEventRecord(fork, cs) == cudaSuccess;
      if (!forked) rc = EFFT_ERR_CUDA;
      for (int g = 1; g < G && forked; ++g)
        if (cudaStreamWaitEvent(side[g], fork, 0) != cudaSuccess) rc = EFFT_ERR_CUDA;
      for (int g = 0; g < G && rc == EFFT_OK && forked; ++g) {
        const int s0 = b->gstart[g], cnt = b->gstart[g + 1] - s0;
        const Batch bt{reinterpret_cast<void* const*>(b->dptrs + s0), (unsigned)cnt, b->state + 4 * (size_t)s0};
        rc = enqueue_batch(b->plans[g], nullptr, bt, g == 0 ? cs : side[g]);
      }
      // join every forked stream, also after an error, so the capture ends cleanly
      for (int g = 1; g < G && forked; ++g)
        if (cudaEventRecord(join[g], side[g]) != cudaSuccess || cudaStreamWaitEvent(cs, join[g], 0) != cudaSuccess)
          if (rc == EFFT_OK) rc = EFFT_ERR_CUDA;
      cudaGraph_t graph = nullptr;
      if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && rc == EFFT_OK) rc = EFFT_ERR_CUDA;
      b->graph = graph;
    }
  }
  if (rc == EFFT_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = EFFT_ERR_CUDA;
  if (rc == EFFT_OK) {
    size_t num = 0;
    if (cudaGraphGetNodes(b->graph, nullptr, &num) == cudaSuccess && num > 0) {
      std::vector<cudaGraphNode_t> nodes(num);
      if (cudaGraphGetNodes(b->graph, nodes.data(), &num) == cudaSuccess)
        for (size_t k = 0; k < num; ++k) {
          cudaGraphNodeType ty;
          if (cudaGraphNodeGetType(nodes[k], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++b->kernels;
        }
    }
  }
  for (int g = 1; g < G; ++g) {
    if (side[g]) cudaStreamDestroy(side[g]);
    if (join[g]) cudaEventDestroy(join[g]);
  }
  if (fork) cudaEventDestroy(fork);
  if (cs) cudaStreamDestroy(cs);
  if (rc != EFFT_OK) cudaGetLastError();
  return rc;
}

}  // namespace

extern "C" {

int efft_batch_create(efft_batch_t* out, const uint64_t* sizes, int count, int dtype, int sign, uint32_t flags) {
  if (!out) return EFFT_ERR_INVALID_PTR;
  *out = nullptr;
  if (!sizes) return EFFT_ERR_INVALID_PTR;
  if (count < 1) return EFFT_ERR_INVALID_SIZE;
  if (dtype != EFFT_C64 && dtype != EFFT_C128) return EFFT_ERR_INVALID_DTYPE;
  if (sign != -1 && sign != 1) return EFFT_ERR_INVALID_SIGN;
  if (flags & ~EFFT_FLAG_ALL) return EFFT_ERR_INVALID_FLAGS;
  std::map<uint64_t, std::vector<int>, std::greater<uint64_t>> by_size;
  for (int i = 0; i < count; ++i) {
    const uint64_t n = sizes[i];
    if (!valid_size(n)) return EFFT_ERR_INVALID_SIZE;
    by_size[n].push_back(i);
  }
  for (auto& kv : by_size)
    if (kv.second.size() > 65535) return EFFT_ERR_INVALID_SIZE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  efft_batch_s* b = new (std::nothrow) efft_batch_s();
  if (!b) return EFFT_ERR_ALLOC;
  b->device = dev;
  b->count = count;
  b->slot.assign(count, 0);
  b->group.assign(count, 0);
  int rc = EFFT_OK;
  int pos = 0;
  for (auto& kv : by_size) {
    const int g = (int)b->plans.size();
    b->gstart.push_back(pos);
    for (int i : kv.second) {
      b->slot[i] = pos++;
      b->group[i] = g;
    }
    efft_plan_t pl = nullptr;
    rc = efft_plan_create(&pl, kv.first, dtype, sign, flags);
    if (rc != EFFT_OK) break;
    b->plans.push_back(pl);
  }
  b->gstart.push_back(count);
  if (rc == EFFT_OK && (cudaMalloc(&b->dptrs, sizeof(void*) * count) != cudaSuccess ||
                        cudaMalloc(&b->state, 16 * (size_t)count) != cudaSuccess ||
                        cudaHostAlloc(&b->stage, sizeof(void*) * count * EFFT_BATCH_INFLIGHT,
                                      cudaHostAllocDefault) != cudaSuccess))
    rc = EFFT_ERR_ALLOC;
  for (int k = 0; rc == EFFT_OK && k < EFFT_BATCH_INFLIGHT; ++k)
    if (cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming) != cudaSuccess) rc = EFFT_ERR_CUDA;
  if (rc == EFFT_OK && cudaMemset(b->dptrs, 0, sizeof(void*) * count) != cudaSuccess) rc = EFFT_ERR_CUDA;
  if (rc == EFFT_OK) rc = batch_capture(b);
  if (rc != EFFT_OK) {
    cudaGetLastError();
    batch_free(b);
    return rc;
  }
  b->magic = kBatchMagic;
  {
    std::lock_guard<std::mutex> lk(registry_mutex());
    if (!g_live_batches) g_live_batches = new std::set<efft_batch_s*>();
    g_live_batches->insert(b);
  }
  *out = b;
  return EFFT_OK;
}

int efft_batch_execute(efft_batch_t b, void* const* data, void* stream) {
  if (!batch_is_live(b)) return EFFT_ERR_INVALID_PLAN;
  if (!data) return EFFT_ERR_INVALID_PTR;
  DeviceGuard g(b->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  // every buffer valid, and no two overlapping (they are transformed concurrently)
  std::vector<std::pair<uintptr_t, uintptr_t>> spans(b->count);
  for (int i = 0; i < b->count; ++i) {
    const efft_plan_s* p = b->plans[b->group[i]];
    int rc = check_buffer(p, data[i]);
    if (rc != EFFT_OK) return rc;
    const uintptr_t a = reinterpret_cast<uintptr_t>(data[i]);
    spans[i] = {a, a + plan_bytes(p)};
  }
  std::sort(spans.begin(), spans.end());
  for (int i = 1; i < b->count; ++i)
    if (spans[i].first < spans[i - 1].second) return EFFT_ERR_INVALID_PTR;
  if (fault_injected("launch")) return EFFT_ERR_LAUNCH;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int k = b->next;
  if (cudaEventSynchronize(b->done[k]) != cudaSuccess) {  // staging slot k free again
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  void** stage = b->stage + (size_t)k * b->count;
  for (int i = 0; i < b->count; ++i) stage[b->slot[i]] = data[i];
  if (cudaMemcpyAsync(b->dptrs, stage, sizeof(void*) * b->count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaGraphLaunch(b->exec, st) != cudaSuccess || cudaEventRecord(b->done[k], st) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_LAUNCH;
  }
  b->next = (k + 1) % EFFT_BATCH_INFLIGHT;
  return EFFT_OK;
}

int efft_batch_info(efft_batch_t b, int* ngroups, int* kernels) {
  if (!batch_is_live(b)) return EFFT_ERR_INVALID_PLAN;
  if (ngroups) *ngroups = (int)b->plans.size();
  if (kernels) *kernels = b->kernels;
  return EFFT_OK;
}

int efft_batch_destroy(efft_batch_t b) {
  if (!b) return EFFT_OK;
  {
    std::lock_guard<std::mutex> lk(registry_mutex());
    if (!g_live_batches || !g_live_batches->count(b) || b->magic != kBatchMagic) return EFFT_ERR_INVALID_PLAN;
    g_live_batches->erase(b);
  }
  b->magic = 0;
  DeviceGuard g(b->device);
  batch_free(b);
  return EFFT_OK;
}

}  // extern "C"
