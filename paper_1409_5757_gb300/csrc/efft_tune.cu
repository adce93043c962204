// efft_tune.cu -- the radix-schedule autotuner (efft_plan_autotune,
// EFFT_FLAG_AUTOTUNE): the GPU counterpart of the paper's scan over the split
// depth s and the worker count (Sec. 5.2, Figs. 6-7).  On a GPU the free
// parameter is the radix schedule, and with it the tile shape of every pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/efft.h"
#include "efft_host.h"

using namespace efft;
using namespace efft::host;

namespace {
// Autotuned schedules per (device, log2 N, dtype).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, Tuned>* g_tuned = nullptr;  // leaked on purpose

}  // namespace

namespace efft {
namespace host {

bool tuned_lookup(int dev, int e, int dtype, Tuned* t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tuned) return false;
  auto it = g_tuned->find(std::make_tuple(dev, e, dtype));
  if (it == g_tuned->end()) return false;
  *t = it->second;
  return true;
}

void tuned_store(int dev, int e, int dtype, const Tuned& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tuned) g_tuned = new std::map<std::tuple<int, int, int>, Tuned>();
  (*g_tuned)[std::make_tuple(dev, e, dtype)] = t;
}

// Every accepted schedule for N = 2^e (at most 1 + 1 + 8 of them).
int schedule_candidates(int e, int (*r)[kMaxPasses], int* np) {
  int k = 0;
  if (e <= 3) {
    np[k++] = 0;
    return k;
  }
  if (e <= 11) {
    r[k][0] = e;
    np[k++] = 1;
  }
  if (e % 2 == 0 && e / 2 >= 4 && e / 2 <= 11) {
    r[k][0] = r[k][1] = e / 2;
    np[k++] = 2;
  }
  for (int a = 4; a <= 11; ++a) {
    const int b = e - 2 * a;
    if (b < 4 || b > 11) continue;
    r[k][0] = r[k][2] = a;
    r[k][1] = b;
    np[k++] = 3;
  }
  return k;
}

int autotune_impl(efft_plan_s* p, void* scratch, cudaStream_t st, int* cand_log2r, double* cand_ms, int cap,
                  int* ncand) {
  int cr[16][kMaxPasses] = {};
  int cnp[16] = {};
  const int nc = schedule_candidates(p->log2n, cr, cnp);
  if (ncand) *ncand = nc;
  int prev_r[kMaxPasses] = {0, 0, 0, 0};
  const int prev_np = p->npasses;
  for (int j = 0; j < prev_np; ++j) prev_r[j] = p->pass[j].log2R;
  const size_t bytes = plan_bytes(p);
  const int reps = (p->n <= (1ull << 20)) ? 21 : (p->n <= (1ull << 26) ? 9 : 5);
  const bool prof = p->profiling;
  p->profiling = false;
  std::vector<cudaEvent_t> ev(2 * reps, nullptr);
  std::vector<float> t(reps, 0.f);
  int rc = EFFT_OK;
  for (auto& x : ev)
    if (cudaEventCreate(&x) != cudaSuccess) {
      rc = EFFT_ERR_CUDA;
      break;
    }
  int best = -1;
  double best_ms = 0.0;
  for (int c = 0; rc == EFFT_OK && c < nc; ++c) {
    apply_schedule(p, cr[c], cnp[c]);
    for (int k = -2; rc == EFFT_OK && k < reps; ++k) {
      // a fresh finite input each time (repeated unnormalised transforms
      // would overflow); the fill is outside the timed interval
      if (cudaMemsetAsync(scratch, 0x3F, bytes, st) != cudaSuccess) {
        rc = EFFT_ERR_LAUNCH;
        break;
      }
      if (k >= 0) cudaEventRecord(ev[2 * k], st);
      rc = enqueue(p, scratch, st);
      if (k >= 0) cudaEventRecord(ev[2 * k + 1], st);
    }
    if (rc != EFFT_OK) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      rc = EFFT_ERR_CUDA;
      break;
    }
    for (int k = 0; k < reps; ++k)
      if (cudaEventElapsedTime(&t[k], ev[2 * k], ev[2 * k + 1]) != cudaSuccess) rc = EFFT_ERR_CUDA;
    if (rc != EFFT_OK) break;
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    const double ms = t[reps / 2];
    if (cand_log2r && c < cap)
      for (int j = 0; j < kMaxPasses; ++j) cand_log2r[kMaxPasses * c + j] = (j < cnp[c]) ? cr[c][j] : 0;
    if (cand_ms && c < cap) cand_ms[c] = ms;
    if (best < 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  for (auto x : ev)
    if (x) cudaEventDestroy(x);
  p->profiling = prof;
  if (rc != EFFT_OK || best < 0) {
    cudaGetLastError();
    apply_schedule(p, prev_r, prev_np);
    return rc == EFFT_OK ? EFFT_ERR_CUDA : rc;
  }
  apply_schedule(p, cr[best], cnp[best]);
  Tuned tu;
  tu.np = cnp[best];
  for (int j = 0; j < kMaxPasses; ++j) tu.r[j] = cr[best][j];
  tuned_store(p->device, p->log2n, p->dtype, tu);
  return EFFT_OK;
}

}  // namespace host
}  // namespace efft

extern "C" {

int efft_plan_autotune(efft_plan_t plan, void* scratch, void* stream, int* cand_log2r, double* cand_ms, int cap,
                       int* ncand) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  DeviceGuard g(plan->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  int rc = check_buffer(plan, scratch);
  if (rc != EFFT_OK) return rc;
  if (plan->real) plan = plan->inner;  // a real plan's schedule is its complex plan's
  if (plan->odd > 1) return EFFT_ERR_UNSUPPORTED;  // N = M * 2^e: one schedule
  return autotune_impl(plan, scratch, reinterpret_cast<cudaStream_t>(stream), cand_log2r, cand_ms,
                       cap < 0 ? 0 : cap, ncand);
}

}  // extern "C"
