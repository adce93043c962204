// efft_host.h -- host-side internals shared by the translation units of
// libefft.so: efft.cu (plans, execution, the C ABI of plans), efft_tune.cu
// (schedule autotuner) and efft_batch.cu (mixed-size batches).  Not part of
// the public interface (include/efft.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/efft.h"
#include "efft_kernels.cuh"

namespace efft {

// The wide complex64 middle pass (R = 2^11, 8 columns) as a persistent
// kernel fed by TMA copies (efft_fx_f32.cu); tensor_map: the array as
// [N / (R s)][R][s] 8-byte elements with 8 x 256 x 1 boxes.
bool fx_launch_f32_mid_tma(dim3 grid, cudaStream_t st, void* data, const PassArgs& a, const void* tensor_map);

namespace host {

constexpr uint32_t kMagic = 0xEFF71409u;
constexpr int kLog2CtaC128 = 12;   // 4096 complex128 elements per CTA (64 KiB)
constexpr int kLog2CtaC64 = 13;    // 8192 complex64 elements per CTA (64 KiB)
constexpr int kMaxPasses = 4;
constexpr int kWideMinLog2N = 28;  // complex128 first passes on 8192-element tiles from 2^28
// complex128 three-pass schedules (a, b, a) with a in 9..11 and b in {8, 10,
// 11} fold the digit swap into the middle pass (and run a strided last pass)
// for 2^26 <= N <= 2^30; measured: 2^28 10.09 vs 11.07 ms, 2^29 22.4 vs
// 23.1, 2^30 44.7 vs 45.3 per transform; from 2^31 on the swapping middle
// pass (one CTA per SM at R = 2^11, or stride 2^21 and more) loses more than
// the swap sweep costs (2^31: 100.2 vs 94.3 ms per step).
constexpr int kFuseMinLog2N = 26;
constexpr int kFuseMaxLog2N = 30;
// complex128 strided passes run persistent, prefetching the next tile, from
// this size on (the wide first pass up to kPersistFirstMaxLog2N)
constexpr int kPersistMinLog2N = 26;
constexpr int kPersistFirstMaxLog2N = 31;
// complex64 wide first pass fed by TMA copies: on wherever the pass shape
// allows it (measured: 2^31 first pass 8.30 ms against 9.16, c4 30.85 ms
// against 31.7; 2^28 1.12 against 1.11)
constexpr bool kTmaRule = true;

// One pass of the schedule and its launch shape.
struct Pass {
  int log2R, log2s, log2L, log2C, kind;
  bool wide;  // complex128 first pass on 8192-element tiles
  int swap;   // middle pass that also swaps the outer digits: log2 of its
              // T x T column tile side (0: no swap)
  bool pf;    // complex128 strided pass run by the persistent prefetching kernel
  bool tma;   // complex64 wide first pass fed by TMA copies (persistent)
  uint64_t grid;
  int threads;
  size_t smem;
  // N = M * 2^e (M > 1): the mixed-radix kernel with integer extents
  bool mixed;
  uint64_t R_int, s_int, L_int;
  int C_int;
  int nrad;
  int rad[8];  // Stockham radices, product R_int
};

// Largest odd factor M of a supported size N = M * 2^e.
constexpr uint32_t kMaxOdd = 15;
// Elements per CTA of the mixed-radix kernel (two padded buffers and the R-th
// roots in shared memory: 100 KiB complex128, 66 KiB complex64).
constexpr int kMixTileC128 = 2048;
constexpr int kMixTileC64 = 2048;

// The transforms one enqueue covers: ptrs (device array of `count` data
// pointers, or NULL for one transform at the enqueue's `data`) and their
// state words (16 bytes per transform).
struct Batch {
  void* const* ptrs;
  unsigned count;
  uint32_t* state;
};

// Range-scan state words of a plan's executes: a ring of kStateRing 16-byte
// words (one per execute) in device memory, each reused only after the
// execute that used it last has finished (an event recorded behind it), so
// that executes of one plan on different buffers need no ordering.
constexpr int kStateRing = 16;
struct StateRing {
  std::mutex mu;
  cudaEvent_t done[kStateRing] = {};
  bool used[kStateRing] = {};
  int next = 0;
};

// Kernel variants of a power-of-two schedule, each -1 (the built-in rule:
// by size), 0 (off) or 1 (on wherever the pass shapes allow it):
//  wide  strided first pass (complex64 also the 2^11 middle pass) on tiles
//        twice as wide (C doubled: longer row segments per page);
//  fuse  complex128 (a, b, a): the middle pass swaps the outer digits and the
//        last pass is strided (no separate swap sweep);
//  pf    complex128 strided passes as persistent kernels that prefetch the
//        next tile.
//  tma   complex64 wide first pass as a persistent kernel fed by TMA copies.
struct Variant {
  int wide = -1, fuse = -1, pf = -1, tma = -1;
};

// A tuned schedule: log2 R_0 .. log2 R_{np-1} and the variant for a power of
// two; for N = M * 2^e the outer radix 2^mixed_a (0: one pass) and the
// variant's tile-width knob.
struct Tuned {
  int np = 0;
  int r[kMaxPasses] = {0, 0, 0, 0};
  Variant v;
  int mixed_a = -1;
};

// Makes `dev` current for the guard's lifetime.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace host
}  // namespace efft

struct efft_plan_s {
  uint32_t magic;
  int device;
  uint64_t n;
  int log2n;
  int dtype;
  int sign;
  uint32_t flags;
  int npasses;
  efft::host::Pass pass[efft::host::kMaxPasses];
  bool small;    // N <= 8: direct-sum kernel
  bool permute;  // final digit swap enabled
  int perm_log2A;     // digit swap: outer extent 2^perm_log2A,
  uint32_t perm_B;    //   middle extent perm_B
  uint32_t odd;       // N = odd * 2^e
  int twB;
  int sms;  // multiprocessors of the plan's device (persistent launches)
  float4* w2048;
  float4* tw_lo;
  float4* tw_hi;
  uint32_t* state;        // kStateRing words of 16 bytes (efft::host::StateRing)
  efft::host::StateRing* ring;
  uint64_t table_bytes;
  // profiling: CUDA event pairs recorded around each launch
  bool profiling;
  struct Rec {
    int slot;
    cudaEvent_t a, b;
  };
  std::vector<Rec>* recs;
  std::vector<cudaEvent_t>* pool;
  // real-data plans (efft_plan_create_real): n reals; the complex work is
  // done by `inner` (n/2 points), the mirrored pairs by efft_real_pairs
  int real;              // 0 complex plan, EFFT_REAL_FORWARD or EFFT_REAL_INVERSE
  efft_plan_s* inner;
  float4* rtw_lo;        // exp(-2*pi*i*t/n), t < 2^rtwB
  float4* rtw_hi;        // exp(-2*pi*i*(t << rtwB)/n), t < (n/2) >> rtwB
  int rtwB;
};

namespace efft {
namespace host {

// The calling thread's device and current context ID (0 when the driver
// cannot report it); makes the device's primary context current.
int current_context(int* dev, unsigned long long* ctx_id);

// Registry of live handles (plans here, batches in efft_batch.cu).
std::mutex& registry_mutex();
bool plan_is_live(efft_plan_s* p);
void register_plan(efft_plan_s* p);
// EFFT_FAULT_INJECT=<what>: host-side failure injection for tests.
bool fault_injected(const char* what);
int ilog2_u64(uint64_t n);
// N = M * 2^e with M odd, M <= kMaxOdd, 1 <= N <= 2^EFFT_MAX_LOG2N.
bool valid_size(uint64_t n);
// Schedule of a plan with N = M * 2^e, M > 1 (pass table and swap); the
// outer radix 2^force_a when force_a >= 0 is a valid choice (0: one pass);
// v.wide >= 0 sets the first pass's tile width instead of the size rule.
int apply_mixed_schedule(efft_plan_s* p, int force_a = -1, const Variant& v = Variant());
// The outer-radix exponents apply_mixed_schedule accepts for p (0: one pass).
int mixed_candidates(const efft_plan_s* p, int* a, int cap);

// Schedules: the planner's table, the accepted set, and filling a plan's
// pass table from a radix list.
int choose_radices(int e, int* r);
bool valid_schedule(int e, const int* r, int np);
int schedule_candidates(int e, int (*r)[kMaxPasses], int* np);
void apply_schedule(efft_plan_s* p, const int* r, int np, const Variant& v = Variant());
// The variant a plan's pass table realises (each knob 0 or 1).
Variant realised_variant(const efft_plan_s* p);
bool tuned_lookup(int dev, uint64_t n, int dtype, Tuned* t);
void tuned_store(int dev, uint64_t n, int dtype, const Tuned& t);

// A plan whose create arguments have been checked; r_explicit != NULL: the
// caller's (validated) schedule.
int plan_create_impl(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags, const int* r_explicit,
                     int np_explicit);
// Times every accepted schedule on `scratch` (then the variants of the
// fastest) and keeps the fastest; out[0..cap) receives the candidates.
int autotune_impl(efft_plan_s* p, void* scratch, cudaStream_t st, efft_candidate* out, int cap, int* ncand);

// Execution: buffer checks and the launch sequence of one transform or of a
// batch of same-size transforms.
int check_buffer(const efft_plan_s* p, const void* data);
// Bytes of the data array of a plan (n complex values, or n reals).
size_t plan_bytes(const efft_plan_s* p);
// Twiddle table generation and the range scan, shared with efft_real.cu.
int gen_table(float4* out, uint64_t count, uint64_t stride, uint64_t N, cudaStream_t st);
int launch_range_scan(const void* data, uint64_t n_complex, uint32_t* state, void* const* ptrs, unsigned count,
                      cudaStream_t st);
void free_plan_memory(efft_plan_s* p);
int prof_begin(efft_plan_s* p, int slot, cudaStream_t st);
void prof_end(efft_plan_s* p, int rec, cudaStream_t st);
// Mixed-radix passes (efft_mix.cu): kernel attributes and one pass launch.
cudaError_t mix_set_attrs();
cudaError_t launch_mix(const efft_plan_s* p, const Pass& ps, void* data, const Batch& bt, cudaStream_t st);
// The real-data launch sequence (efft_real.cu).
// `state`: the execute's 16-byte device state word.
int enqueue_real(efft_plan_s* p, void* data, uint32_t* state, cudaStream_t st);
int enqueue_batch(efft_plan_s* p, void* data, const Batch& bt, cudaStream_t st);
// One transform with the given state word (the caller owns its ordering).
int enqueue_state(efft_plan_s* p, void* data, uint32_t* state, cudaStream_t st);
// One transform with a state word of the plan's ring (or, while `st` is
// being captured into a CUDA graph, one allocated in that graph).
int enqueue(efft_plan_s* p, void* data, cudaStream_t st);
// Device state of a plan: kStateRing zeroed words and their events.
int ring_create(efft_plan_s* p, cudaStream_t st);

}  // namespace host
}  // namespace efft
