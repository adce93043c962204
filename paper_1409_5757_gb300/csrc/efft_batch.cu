// efft_batch.cu -- batches of independent in-place transforms of mixed
// sizes behind one CUDA graph (efft_batch_* in include/efft.h), and host data
// through a chain of batches with the copies overlapped.
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

// Host data through a chain of batches of the same sizes: the transforms are
// taken group by group (largest size first) in chunks of about
// kHostChunkBytes; a chunk's copies in, its launches for every batch of the
// chain and its copies out run on three streams ordered by events, so the
// copies of one chunk overlap the transforms of the previous ones.
int efft_batch_execute_host_stream(const efft_batch_t* batches, int nbatches, void* const* host_in,
                                   void* const* host_out, void* const* dev, void* stream) {
  constexpr size_t kHostChunkBytes = 256ull << 20;
  if (!batches || nbatches < 1) return EFFT_ERR_INVALID_SIZE;
  for (int j = 0; j < nbatches; ++j)
    if (!batch_is_live(batches[j])) return EFFT_ERR_INVALID_PLAN;
  efft_batch_s* b0 = batches[0];
  // every batch of the chain: same device, dtype, sizes and slot layout
  for (int j = 1; j < nbatches; ++j) {
    const efft_batch_s* b = batches[j];
    if (b->device != b0->device || b->count != b0->count || b->gstart != b0->gstart || b->slot != b0->slot ||
        b->plans.size() != b0->plans.size())
      return EFFT_ERR_INVALID_SIZE;
    for (size_t g = 0; g < b->plans.size(); ++g)
      if (b->plans[g]->n != b0->plans[g]->n || b->plans[g]->dtype != b0->plans[g]->dtype)
        return EFFT_ERR_INVALID_SIZE;
  }
  if (!host_in || !host_out || !dev) return EFFT_ERR_INVALID_PTR;
  const int count = b0->count;
  DeviceGuard dg(b0->device);
  if (!dg.ok) return EFFT_ERR_CUDA;
  std::vector<std::pair<uintptr_t, uintptr_t>> spans(count);
  std::vector<int> by_slot(count);
  for (int i = 0; i < count; ++i) {
    if (!host_in[i] || !host_out[i]) return EFFT_ERR_INVALID_PTR;
    const efft_plan_s* p = b0->plans[b0->group[i]];
    int rc = check_buffer(p, dev[i]);
    if (rc != EFFT_OK) return rc;
    const uintptr_t a = reinterpret_cast<uintptr_t>(dev[i]);
    spans[i] = {a, a + plan_bytes(p)};
    by_slot[b0->slot[i]] = i;
  }
  std::sort(spans.begin(), spans.end());
  for (int i = 1; i < count; ++i)
    if (spans[i].first < spans[i - 1].second) return EFFT_ERR_INVALID_PTR;
  if (fault_injected("launch")) return EFFT_ERR_LAUNCH;

  // chunks: runs of slots inside one group of about kHostChunkBytes
  struct Chunk {
    int g, s0, s1;
  };
  std::vector<Chunk> chunks;
  for (size_t g = 0; g + 1 < b0->gstart.size(); ++g) {
    const size_t bytes = plan_bytes(b0->plans[g]);
    const int per = (int)std::max<size_t>(1, kHostChunkBytes / bytes);
    for (int s = b0->gstart[g]; s < b0->gstart[g + 1]; s += per)
      chunks.push_back({(int)g, s, std::min(s + per, b0->gstart[g + 1])});
  }

  cudaStream_t sc = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t sin = nullptr, sout = nullptr;
  std::vector<cudaEvent_t> ev_in(chunks.size(), nullptr), ev_comp(chunks.size(), nullptr);
  int rc = EFFT_OK;
  if (cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking) != cudaSuccess)
    rc = EFFT_ERR_CUDA;
  for (size_t c = 0; rc == EFFT_OK && c < chunks.size(); ++c)
    if (cudaEventCreateWithFlags(&ev_in[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_comp[c], cudaEventDisableTiming) != cudaSuccess)
      rc = EFFT_ERR_CUDA;
  // the pointer arrays of every batch (staging slots as in efft_batch_execute)
  std::vector<int> ring(nbatches, 0);
  for (int j = 0; rc == EFFT_OK && j < nbatches; ++j) {
    efft_batch_s* b = batches[j];
    const int k = b->next;
    if (cudaEventSynchronize(b->done[k]) != cudaSuccess) {
      rc = EFFT_ERR_CUDA;
      break;
    }
    void** stage = b->stage + (size_t)k * count;
    for (int i = 0; i < count; ++i) stage[b->slot[i]] = dev[i];
    if (cudaMemcpyAsync(b->dptrs, stage, sizeof(void*) * count, cudaMemcpyHostToDevice, sc) != cudaSuccess)
      rc = EFFT_ERR_CUDA;
    ring[j] = k;
    b->next = (k + 1) % EFFT_BATCH_INFLIGHT;
  }
  for (size_t c = 0; rc == EFFT_OK && c < chunks.size(); ++c) {
    const Chunk& ch = chunks[c];
    const size_t bytes = plan_bytes(b0->plans[ch.g]);
    for (int s = ch.s0; rc == EFFT_OK && s < ch.s1; ++s) {
      const int i = by_slot[s];
      if (cudaMemcpyAsync(dev[i], host_in[i], bytes, cudaMemcpyHostToDevice, sin) != cudaSuccess) rc = EFFT_ERR_CUDA;
    }
    if (rc != EFFT_OK || cudaEventRecord(ev_in[c], sin) != cudaSuccess ||
        cudaStreamWaitEvent(sc, ev_in[c], 0) != cudaSuccess) {
      rc = EFFT_ERR_CUDA;
      break;
    }
    for (int j = 0; rc == EFFT_OK && j < nbatches; ++j) {
      efft_batch_s* b = batches[j];
      const Batch bt{reinterpret_cast<void* const*>(b->dptrs + ch.s0), (unsigned)(ch.s1 - ch.s0),
                     b->state + 4 * (size_t)ch.s0};
      rc = enqueue_batch(b->plans[ch.g], nullptr, bt, sc);
    }
    if (rc != EFFT_OK) break;
    if (cudaEventRecord(ev_comp[c], sc) != cudaSuccess || cudaStreamWaitEvent(sout, ev_comp[c], 0) != cudaSuccess) {
      rc = EFFT_ERR_CUDA;
      break;
    }
    for (int s = ch.s0; rc == EFFT_OK && s < ch.s1; ++s) {
      const int i = by_slot[s];
      if (cudaMemcpyAsync(host_out[i], dev[i], bytes, cudaMemcpyDeviceToHost, sout) != cudaSuccess) rc = EFFT_ERR_CUDA;
    }
  }
  for (int j = 0; j < nbatches; ++j) cudaEventRecord(batches[j]->done[ring[j]], sc);
  // drain everything that was enqueued, even after an error
  if (sin) cudaStreamSynchronize(sin);
  cudaStreamSynchronize(sc);
  if (sout && cudaStreamSynchronize(sout) != cudaSuccess && rc == EFFT_OK) rc = EFFT_ERR_CUDA;
  for (size_t c = 0; c < chunks.size(); ++c) {
    if (ev_in[c]) cudaEventDestroy(ev_in[c]);
    if (ev_comp[c]) cudaEventDestroy(ev_comp[c]);
  }
  if (sin) cudaStreamDestroy(sin);
  if (sout) cudaStreamDestroy(sout);
  if (rc != EFFT_OK) cudaGetLastError();
  return rc;
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
