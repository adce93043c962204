// efft_tune.cu -- the schedule autotuner (efft_plan_autotune,
// EFFT_FLAG_AUTOTUNE): the GPU counterpart of the paper's scan over the split
// depth s and the worker count (Sec. 5.2, Figs. 6-7).  On a GPU the free
// parameters are the radix schedule (for N = M * 2^e the outer radix of the
// (2^a, M * 2^b, 2^a) schedule) and the kernel variant of its passes: the
// tile width of the strided passes (C doubled or not), the digit swap folded
// into the middle pass or not, the persistent prefetching pass kernels or
// not, and the TMA-fed complex64 passes or not (N = M * 2^e: the tile width
// of the first pass only).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/efft.h"
#include "efft_host.h"

using namespace efft;
using namespace efft::host;

namespace {
// Tuned schedules per (device, N, dtype).
std::mutex g_tune_mu;
std::map<std::tuple<int, uint64_t, int>, Tuned>* g_tuned = nullptr;  // leaked on purpose

// What a candidate runs: a power-of-two schedule with a variant, or for
// N = M * 2^e an outer radix.
struct Cand {
  Tuned t;
};

void apply(efft_plan_s* p, const Tuned& t) {
  if (p->odd > 1) apply_mixed_schedule(p, t.mixed_a, t.v);
  else apply_schedule(p, t.r, t.np, t.v);
}

// The record of a candidate as the plan now runs it.
efft_candidate describe(const efft_plan_s* p, double ms) {
  efft_candidate c;
  std::memset(&c, 0, sizeof(c));
  c.npasses = p->npasses;
  for (int j = 0; j < p->npasses && j < 4; ++j)
    c.radices[j] = p->pass[j].mixed ? p->pass[j].R_int : (1ull << p->pass[j].log2R);
  const Variant v = realised_variant(p);
  c.wide = v.wide;
  c.fused_swap = v.fuse;
  c.persistent = v.pf;
  c.tma = v.tma;
  c.ms = ms;
  return c;
}

// A signature of the pass table: two candidates with the same signature run
// the same launches.
std::vector<int> signature(const efft_plan_s* p) {
  std::vector<int> s = {p->npasses, p->permute ? 1 : 0};
  for (int j = 0; j < p->npasses; ++j) {
    const Pass& q = p->pass[j];
    s.insert(s.end(), {q.kind, q.log2R, q.log2C, q.wide ? 1 : 0, q.swap, q.pf ? 1 : 0, q.tma ? 1 : 0, (int)q.R_int});
  }
  return s;
}

}  // namespace

namespace efft {
namespace host {

bool tuned_lookup(int dev, uint64_t n, int dtype, Tuned* t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tuned) return false;
  auto it = g_tuned->find(std::make_tuple(dev, n, dtype));
  if (it == g_tuned->end()) return false;
  *t = it->second;
  return true;
}

void tuned_store(int dev, uint64_t n, int dtype, const Tuned& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tuned) g_tuned = new std::map<std::tuple<int, uint64_t, int>, Tuned>();
  (*g_tuned)[std::make_tuple(dev, n, dtype)] = t;
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

int autotune_impl(efft_plan_s* p, void* scratch, cudaStream_t st, efft_candidate* out, int cap, int* ncand) {
  // the plan's current choice, restored on failure
  Tuned prev;
  if (p->odd > 1) {
    prev.mixed_a = -1;
    if (p->npasses == 3) prev.mixed_a = __builtin_ctzll(p->pass[0].mixed ? p->pass[0].R_int : (1ull << p->pass[0].log2R));
    else prev.mixed_a = 0;
  } else {
    prev.np = p->npasses;
    for (int j = 0; j < prev.np; ++j) prev.r[j] = p->pass[j].log2R;
  }
  prev.v = realised_variant(p);
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
  int count = 0;
  // median time of one execute with the plan as it stands
  auto measure = [&](double* ms) -> int {
    for (int k = -2; k < reps; ++k) {
      // a fresh finite input each time (repeated unnormalised transforms
      // would overflow); the fill is outside the timed interval
      if (cudaMemsetAsync(scratch, 0x3F, bytes, st) != cudaSuccess) return EFFT_ERR_LAUNCH;
      if (k >= 0) cudaEventRecord(ev[2 * k], st);
      const int r = enqueue(p, scratch, st);
      if (r != EFFT_OK) return r;
      if (k >= 0) cudaEventRecord(ev[2 * k + 1], st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return EFFT_ERR_CUDA;
    for (int k = 0; k < reps; ++k)
      if (cudaEventElapsedTime(&t[k], ev[2 * k], ev[2 * k + 1]) != cudaSuccess) return EFFT_ERR_CUDA;
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    *ms = t[reps / 2];
    return EFFT_OK;
  };
  auto record = [&](double ms) {
    if (out && count < cap) out[count] = describe(p, ms);
    ++count;
  };

  Tuned best;
  double best_ms = -1.0;
  // 1. schedules (power of two: with the size rules for the variant)
  std::vector<Tuned> cands;
  if (p->odd > 1) {
    int as[32];
    const int na = std::min(mixed_candidates(p, as, 32), 32);
    for (int i = 0; i < na; ++i) {
      Tuned c;
      c.mixed_a = as[i];
      cands.push_back(c);
    }
  } else {
    int cr[16][kMaxPasses] = {};
    int cnp[16] = {};
    const int nc = schedule_candidates(p->log2n, cr, cnp);
    for (int i = 0; i < nc; ++i) {
      Tuned c;
      c.np = cnp[i];
      for (int j = 0; j < kMaxPasses; ++j) c.r[j] = cr[i][j];
      cands.push_back(c);
    }
  }
  for (size_t i = 0; rc == EFFT_OK && i < cands.size(); ++i) {
    apply(p, cands[i]);
    double ms = 0.0;
    rc = measure(&ms);
    if (rc != EFFT_OK) break;
    record(ms);
    if (best_ms < 0 || ms < best_ms) {
      best = cands[i];
      best.v = realised_variant(p);
      best_ms = ms;
    }
  }
  // 2. each variant knob of the fastest schedule switched the other way,
  // where that changes the launches; kept when faster (N = M * 2^e: the
  // first pass's tile width only)
  const int nknobs = (p->odd > 1) ? 1 : 4;
  for (int knob = 0; rc == EFFT_OK && best_ms >= 0 && knob < nknobs; ++knob) {
    Tuned c = best;
    int* k = (knob == 0) ? &c.v.wide : (knob == 1) ? &c.v.fuse : (knob == 2) ? &c.v.pf : &c.v.tma;
    apply(p, best);
    const std::vector<int> s0 = signature(p);
    *k = 1 - *k;
    apply(p, c);
    if (signature(p) == s0) continue;
    c.v = realised_variant(p);
    double ms = 0.0;
    rc = measure(&ms);
    if (rc != EFFT_OK) break;
    record(ms);
    if (ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  for (auto x : ev)
    if (x) cudaEventDestroy(x);
  p->profiling = prof;
  if (ncand) *ncand = count;
  if (rc != EFFT_OK || best_ms < 0) {
    cudaGetLastError();
    apply(p, prev);
    return rc == EFFT_OK ? EFFT_ERR_CUDA : rc;
  }
  apply(p, best);
  tuned_store(p->device, p->n, p->dtype, best);
  return EFFT_OK;
}

}  // namespace host
}  // namespace efft

extern "C" {

int efft_plan_autotune_candidates(efft_plan_t plan, void* scratch, void* stream, efft_candidate* out, int cap,
                                  int* ncand) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  DeviceGuard g(plan->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  int rc = check_buffer(plan, scratch);
  if (rc != EFFT_OK) return rc;
  if (plan->real) plan = plan->inner;  // a real plan's schedule is its complex plan's
  return autotune_impl(plan, scratch, reinterpret_cast<cudaStream_t>(stream), out, cap < 0 ? 0 : cap, ncand);
}

int efft_plan_autotune(efft_plan_t plan, void* scratch, void* stream, int* cand_log2r, double* cand_ms, int cap,
                       int* ncand) {
  if (cap < 0) cap = 0;
  std::vector<efft_candidate> rec((size_t)cap);
  int n = 0;
  const int rc = efft_plan_autotune_candidates(plan, scratch, stream, cap ? rec.data() : nullptr, cap, &n);
  if (ncand) *ncand = n;
  for (int c = 0; c < cap && c < n; ++c) {
    for (int j = 0; j < kMaxPasses; ++j)
      if (cand_log2r)
        cand_log2r[kMaxPasses * c + j] = (j < rec[c].npasses) ? __builtin_ctzll(rec[c].radices[j]) : 0;
    if (cand_ms) cand_ms[c] = rec[c].ms;
  }
  return rc;
}

int efft_plan_set_variant(efft_plan_t plan, int wide, int fused_swap, int persistent, int tma) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (plan->real) plan = plan->inner;
  for (int k : {wide, fused_swap, persistent, tma})
    if (k < -1 || k > 1) return EFFT_ERR_INVALID_FLAGS;
  if (plan->odd > 1) {
    // N = M * 2^e: the first pass's tile width only
    if (fused_swap != -1 || persistent != -1 || tma != -1) return EFFT_ERR_UNSUPPORTED;
    Variant v;
    v.wide = wide;
    const int a = (plan->npasses == 3) ? __builtin_ctzll(plan->pass[0].mixed ? plan->pass[0].R_int
                                                                               : (1ull << plan->pass[0].log2R))
                                       : 0;
    return apply_mixed_schedule(plan, a, v);
  }
  Variant v;
  v.wide = wide;
  v.fuse = fused_swap;
  v.pf = persistent;
  v.tma = tma;
  int r[kMaxPasses] = {0, 0, 0, 0};
  const int np = plan->npasses;
  for (int j = 0; j < np; ++j) r[j] = plan->pass[j].log2R;
  apply_schedule(plan, r, np, v);
  return EFFT_OK;
}

int efft_plan_variant(efft_plan_t plan, int* wide, int* fused_swap, int* persistent, int* tma) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (plan->real) plan = plan->inner;
  const Variant v = realised_variant(plan);
  if (wide) *wide = v.wide;
  if (fused_swap) *fused_swap = v.fuse;
  if (persistent) *persistent = v.pf;
  if (tma) *tma = v.tma;
  return EFFT_OK;
}

}  // extern "C"
