// efft.cu -- plan creation, pass schedule and the C ABI of include/efft.h.
//
// Host side of the in-place multi-pass DFT.  A plan fixes the radices
// N = R_0 * ... * R_{p-1} (the paper's splits, Sec. 3, restated as
// mixed-radix passes), owns the O(sqrt N) twiddle tables that the paper's
// constructor precomputes once (Sec. 3.1, Listing 3) and a 16-byte state
// word; an execute enqueues the pass kernels on the caller's stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "../../include/efft.h"
#include "efft_host.h"
#include "efft_kernels.cuh"

using namespace efft;
using namespace efft::host;

namespace efft {
// ----------------------------------------------------------------------------
// Range scan: largest biased binary64 exponent among all re/im parts.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) efft_range_scan(const uint4* __restrict__ x, uint64_t n,
                                                        uint32_t* __restrict__ state, void* const* ptrs) {
  if (ptrs) {  // batched launch: transform blockIdx.y
    x = reinterpret_cast<const uint4*>(ptrs[blockIdx.y]);
    state += 4u * blockIdx.y;
  }
  uint32_t mx = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    uint4 v0 = __ldg(x + i), v1 = __ldg(x + i + stride), v2 = __ldg(x + i + 2 * stride),
          v3 = __ldg(x + i + 3 * stride);
    mx = max(mx, max(max(v0.y & 0x7FF00000u, v0.w & 0x7FF00000u), max(v1.y & 0x7FF00000u, v1.w & 0x7FF00000u)));
    mx = max(mx, max(max(v2.y & 0x7FF00000u, v2.w & 0x7FF00000u), max(v3.y & 0x7FF00000u, v3.w & 0x7FF00000u)));
  }
  for (; i < n; i += stride) {
    uint4 v = __ldg(x + i);
    mx = max(mx, max(v.y & 0x7FF00000u, v.w & 0x7FF00000u));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  __shared__ uint32_t wmax[8];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, wmax[w]);
    atomicMax(state, r >> 20);
  }
}

// ----------------------------------------------------------------------------
// In-place digit reversal for radices (a, b, a) (the scatter of Sec. 3.2,
// done as pairwise tile swaps): position (i0, i1, i2) with
// i0, i2 < A, i1 < B swaps with (i2, i1, i0).  For fixed i1 this is the
// transpose of an A x A matrix with row stride B*A; CTA z handles the tile
// pair (I, J), (J, I) with I <= J (triangular decode of blockIdx.x).
// T x T tiles, T = min(32, A); 256 threads.
// ----------------------------------------------------------------------------
template <typename E>
__global__ void __launch_bounds__(256) efft_digit_swap(E* __restrict__ data, int log2A, uint32_t B, int log2T,
                                                       E* const* ptrs) {
  if (ptrs) data = ptrs[blockIdx.z];  // batched launch: transform blockIdx.z
  __shared__ E t0[32][33];
  __shared__ E t1[32][33];
  const int T = 1 << log2T;
  const uint64_t A = 1ull << log2A;
  const uint64_t rowstride = A * B;  // stride of i0 (B = extent of the middle digit)
  const uint64_t i1 = blockIdx.y;
  // triangular decode: z -> (I, J), I <= J
  const uint32_t z = blockIdx.x;
  uint32_t J = (uint32_t)((sqrtf(8.0f * (float)z + 1.0f) - 1.0f) * 0.5f);
  while ((J + 1) * (J + 2) / 2 <= z) ++J;
  while (J * (J + 1) / 2 > z) --J;
  const uint32_t I = z - J * (J + 1) / 2;
  const uint64_t base = i1 << log2A;
  // tile (I, J): rows i0 = I*T + r, cols i2 = J*T + col
  if (sizeof(E) == 8 && log2T == 5 && blockDim.x == 256) {
    // 32 x 32 tiles of 8-byte elements: each thread's four elements of each
    // tile are loaded before any is stored, eight loads in flight per thread
    // (complex64 2^31: 5.73 -> 4.97 ms; the same for 16-byte elements
    // measured slower, 46.8 -> 47.9 ms at complex128 2^33)
    E a0[4], a1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q, r = e >> 5, col = e & 31;
      a0[q] = data[base + ((uint64_t)I * 32 + r) * rowstride + (uint64_t)J * 32 + col];
      if (I != J) a1[q] = data[base + ((uint64_t)J * 32 + r) * rowstride + (uint64_t)I * 32 + col];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q, r = e >> 5, col = e & 31;
      t0[r][col] = a0[q];
      if (I != J) t1[r][col] = a1[q];
    }
  } else {
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      int r = e >> log2T, col = e & (T - 1);
      t0[r][col] = data[base + ((uint64_t)I * T + r) * rowstride + (uint64_t)J * T + col];
      if (I != J) t1[r][col] = data[base + ((uint64_t)J * T + r) * rowstride + (uint64_t)I * T + col];
    }
  }
  __syncthreads();
  // position (J*T + r, i1, I*T + col) receives old (I*T + col, i1, J*T + r) = t0[col][r]
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    int r = e >> log2T, col = e & (T - 1);
    data[base + ((uint64_t)J * T + r) * rowstride + (uint64_t)I * T + col] = t0[col][r];
    if (I != J) data[base + ((uint64_t)I * T + r) * rowstride + (uint64_t)J * T + col] = t1[col][r];
  }
}

// ----------------------------------------------------------------------------
// Twiddle tables: out[t] = exp(-2*pi*i * t*stride / N) for t < count, FP64
// sincospi of the phase reduced mod N in integers (exact for N a power of
// two; for N = M * 2^e the quotient is rounded once), split into FP32
// (hi, lo).
// ----------------------------------------------------------------------------
__global__ void efft_twiddles(float4* __restrict__ out, uint64_t count, uint64_t stride, uint64_t N) {
  uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint64_t mN = (N & (N - 1)) ? (t * stride) % N : (t * stride) & (N - 1);
  const double x = -2.0 * ((double)mN / (double)N);
  double sv, cv;
  sincospi(x, &sv, &cv);
  float ch = __double2float_rn(cv), sh = __double2float_rn(sv);
  float cl = __double2float_rn(cv - (double)ch), sl = __double2float_rn(sv - (double)sh);
  out[t] = make_float4(ch, cl, sh, sl);
}

}  // namespace efft

namespace {
constexpr size_t kCopyChunk = size_t(1) << 30;  // host copies of the streaming entry point
std::mutex g_mu;
}  // namespace

namespace efft {
namespace host {

std::mutex& registry_mutex() { return g_mu; }

std::set<efft_plan_s*>* g_live = nullptr;  // leaked on purpose: safe at exit

bool plan_is_live(efft_plan_s* p) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_live && g_live->count(p) && p->magic == kMagic;
}

void register_plan(efft_plan_s* p) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_live) g_live = new std::set<efft_plan_s*>();
  g_live->insert(p);
}

bool fault_injected(const char* what) {
  const char* v = std::getenv("EFFT_FAULT_INJECT");
  return v && std::strcmp(v, what) == 0;
}

int ilog2_u64(uint64_t n) {
  int e = 0;
  while ((1ull << e) < n) ++e;
  return e;
}

bool valid_size(uint64_t n) {
  if (n == 0 || n > (1ull << EFFT_MAX_LOG2N)) return false;
  const uint64_t odd = n / (n & (~n + 1));
  return odd <= kMaxOdd;
}

// N = M * 2^e, M > 1: one mixed-radix pass when N fits a CTA, else three
// passes (A, B, A) with A = 2^a and B = M * 2^(e - 2a) (palindromic, so the
// digit reversal is still the swap of the outer digits), choosing a to make
// the larger of A and B smallest.
// Whether (2^a, M * 2^b, 2^a) (a >= 1), or one pass (a = 0), is a schedule
// the mixed-radix kernels run for p.
static bool mixed_ok(const efft_plan_s* p, int a) {
  const uint64_t n = p->n;
  const int tile = (p->dtype == EFFT_C128) ? kMixTileC128 : kMixTileC64;
  const int e = __builtin_ctzll(n);
  if (a == 0) return n <= (uint64_t)tile;
  if (2 * a > e) return false;
  const uint64_t A = 1ull << a, B = n / (A * A);
  return A <= (uint64_t)tile && B <= (uint64_t)tile;
}

// An explicit schedule for N = M * 2^e, M > 1: one pass (log2 R_0 = e, N
// within a CTA tile) or (2^a, M * 2^b, 2^a) given as (a, b, a).
static bool valid_mixed_schedule(uint64_t n, int dtype, const int* r, int np) {
  efft_plan_s q;
  std::memset(&q, 0, sizeof(q));
  q.n = n;
  q.dtype = dtype;
  const int e = __builtin_ctzll(n);
  if (!r) return false;
  if (np == 1) return r[0] == e && mixed_ok(&q, 0);
  return np == 3 && r[0] >= 1 && r[0] == r[2] && r[1] >= 0 && 2 * r[0] + r[1] == e && mixed_ok(&q, r[0]);
}

int mixed_candidates(const efft_plan_s* p, int* a, int cap) {
  int k = 0;
  for (int c = 0; 2 * c <= __builtin_ctzll(p->n); ++c)
    if (mixed_ok(p, c)) {
      if (k < cap) a[k] = c;
      ++k;
    }
  return k;
}

int apply_mixed_schedule(efft_plan_s* p, int force_a, const Variant& v) {
  const uint64_t n = p->n;
  const int tile = (p->dtype == EFFT_C128) ? kMixTileC128 : kMixTileC64;
  const size_t eb = (p->dtype == EFFT_C128) ? 16 : 8;
  const int e = __builtin_ctzll(n);
  int np = 1, a = 0;
  if (force_a >= 0 && mixed_ok(p, force_a)) {
    a = force_a;
    np = (a == 0) ? 1 : 3;
  } else if (n > (uint64_t)tile) {
    // the largest A whose middle radix B = M * 2^b keeps b >= 4 (the
    // compile-time middle-pass kernel): the power-of-two outer passes are
    // the efficient ones; failing that, the A minimising the larger radix.
    // A <= 2^11 for complex128, <= 2^10 for complex64 (its radix-32 kernels)
    const uint64_t amax = (p->dtype == EFFT_C128) ? 2048 : 1024;
    for (int c = 1; 2 * c <= e; ++c) {
      const uint64_t A = 1ull << c, B = n / (A * A);
      if (A > amax || A > (uint64_t)tile || B > (uint64_t)tile) continue;
      if (__builtin_ctzll(B) >= 4) a = c;
    }
    uint64_t best = 0;
    for (int c = 1; a == 0 && 2 * c <= e; ++c) {
      const uint64_t A = 1ull << c, B = n / (A * A);
      if (A > (uint64_t)tile || B > (uint64_t)tile) continue;
      const uint64_t big = A > B ? A : B;
      if (best == 0 || big < best) {
        best = big;
        a = c;
      }
    }
    if (a == 0) return EFFT_ERR_UNSUPPORTED;
    np = 3;
  }
  const uint64_t A = 1ull << a, B = (np == 3) ? n / (A * A) : n;
  const uint64_t Rs[3] = {np == 3 ? A : n, B, A};
  const uint64_t ss[3] = {np == 3 ? n / A : 1, A, 1};
  const uint64_t Ls[3] = {n, A * B, A};
  p->npasses = np;
  p->small = false;
  for (int j = 0; j < kMaxPasses; ++j) p->pass[j] = Pass();
  for (int j = 0; j < np; ++j) {
    Pass& ps = p->pass[j];
    const int jj = (np == 1) ? 0 : j;
    ps.mixed = true;
    ps.R_int = (np == 1) ? n : Rs[jj];
    ps.s_int = (np == 1) ? 1 : ss[jj];
    ps.L_int = (np == 1) ? n : Ls[jj];
    ps.kind = (np == 1) ? SINGLE : (j == 0 ? FIRST : (j == 1 ? MID : LAST));
    ps.log2R = __builtin_ctzll(ps.R_int);  // the power-of-two part (efft_plan_radices)
    // Stockham radices: the odd factor, then 16s, then one 8, 4 or 2
    uint64_t rest = ps.R_int;
    ps.nrad = 0;
    const uint64_t odd = rest / (rest & (~rest + 1));
    if (odd > 1) {
      ps.rad[ps.nrad++] = (int)odd;
      rest /= odd;
    }
    while (rest % 16 == 0) {
      ps.rad[ps.nrad++] = 16;
      rest /= 16;
    }
    if (rest > 1) ps.rad[ps.nrad++] = (int)rest;
    // columns per CTA: a power of two dividing the stride (a CTA's columns
    // stay inside one block) and the column count
    const uint64_t ncol = n / ps.R_int;
    int C = 1;
    while ((uint64_t)(2 * C) * ps.R_int <= (uint64_t)tile && ncol % (uint64_t)(2 * C) == 0 &&
           (ps.s_int == 1 || ps.s_int % (uint64_t)(2 * C) == 0))
      C *= 2;
    ps.C_int = C;
    ps.grid = ncol / (uint64_t)C;
    ps.threads = 256;
    const size_t cr = (size_t)C * ps.R_int;
    ps.smem = 2 * (cr + cr / 16) * eb + ps.R_int * sizeof(float4);  // two padded buffers, the R-th roots
    // outer passes of radix 2^8..2^11: the specialised power-of-two kernels
    // (the first pass with stride M * 2^(e-a), the last on contiguous blocks)
    if (np == 3 && j != 1 && a >= 8 && a <= 11) {
      const int log2cta = (p->dtype == EFFT_C128) ? kLog2CtaC128 : kLog2CtaC64;
      ps.mixed = false;
      ps.log2s = (j == 0) ? e - a : 0;
      ps.log2L = ps.log2s + a;
      // the first pass's tile width: the size rule, or the variant's knob
      const bool wide_on = (v.wide < 0) ? n >= (1ull << kWideMinLog2N) : v.wide != 0;
      ps.wide = j == 0 && wide_on && (p->dtype == EFFT_C128 ? a >= 10 : a == 10);
      ps.log2C = (ps.wide ? (p->dtype == EFFT_C128 ? kLog2CtaWide : kLog2CtaWideC64) : log2cta) - a;
      ps.grid = ncol >> ps.log2C;
      ps.threads = 1 << (a + ps.log2C - 4);
      const size_t elems = 1ull << (a + ps.log2C);
      ps.smem = (elems + elems / 16 + 1) * eb;
    }
  }
  p->permute = (np == 3) && !(p->flags & EFFT_FLAG_DIGIT_REVERSED_OUT);
  p->perm_log2A = (np == 3) ? a : 0;
  p->perm_B = (np == 3) ? (uint32_t)B : 1u;
  return EFFT_OK;
}

// Radix schedule.  Symmetric radix lists (R_j = R_{p-1-j}) make the final
// digit reversal an involution, so it can be done in place by tile swaps.
// For three passes (a, b, a) the table prefers radices 2^8..2^11 (the
// specialised kernels), few internal stages (2^8 = 16*16 is the cheapest per
// bit) and, once the array is large, at most 2^10 rows in the first pass: its
// columns span the whole array, and 2^11 rows at page-sized strides exceed
// the GPU's address-translation reach (measured: 2^30 with (10,10,10) runs
// 10% faster than (11,8,11)).  2^32 and 2^33 need 2^11 in the first pass.
int choose_radices(int e, int* r) {
  if (e <= 3) return 0;  // handled by the direct-sum kernel (or identity)
  if (e <= 11) { r[0] = e; return 1; }
  if (e <= 22 && (e % 2) == 0) { r[0] = r[1] = e / 2; return 2; }
  static const int kA[34] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
                             /*13*/ 4, 0, /*15*/ 5, 0, /*17*/ 6, 0, /*19*/ 7, 0, /*21*/ 8, 0,
                             /*23*/ 8, 8, 8, 8, 8, /*28*/ 10, /*29*/ 9, /*30*/ 10, /*31*/ 10, /*32*/ 11, /*33*/ 11};
  const int a = kA[e];
  r[0] = r[2] = a;
  r[1] = e - 2 * a;
  return 3;
}

// A radix list the kernels accept: none for N <= 8; one pass of 2^4..2^11;
// two or three passes of 2^4..2^11 each, symmetric (R_0 = R_{p-1}).
bool valid_schedule(int e, const int* r, int np) {
  if (e <= 3) return np == 0;
  if (np < 1 || np > 3 || !r) return false;
  int sum = 0;
  for (int j = 0; j < np; ++j) {
    if (r[j] < 4 || r[j] > 11) return false;
    sum += r[j];
  }
  return sum == e && r[0] == r[np - 1];
}

// Fills the pass table of p (log2n, dtype and flags already set) for the
// radix list r[0..np) and the kernel variant v (-1 knobs: the size rules).
void apply_schedule(efft_plan_s* p, const int* r, int np, const Variant& v) {
  const int e = p->log2n;
  const bool c128 = (p->dtype == EFFT_C128);
  auto on = [](int knob, bool rule) { return knob < 0 ? rule : knob != 0; };
  const bool wide_on = on(v.wide, e >= kWideMinLog2N) && e >= (c128 ? kLog2CtaWide : kLog2CtaWideC64);
  const bool fuse_on = on(v.fuse, e >= kFuseMinLog2N && e <= kFuseMaxLog2N);
  const int pf = v.pf;  // -1: per-pass rules below
  p->npasses = np;
  p->small = (e >= 1 && e <= 3);
  const int log2cta = c128 ? kLog2CtaC128 : kLog2CtaC64;
  const size_t eb = c128 ? 16 : 8;
  int rest = e;
  for (int j = 0; j < kMaxPasses; ++j) p->pass[j] = Pass();
  for (int j = 0; j < np; ++j) {
    Pass& ps = p->pass[j];
    ps.log2R = r[j];
    rest -= r[j];
    ps.log2s = rest;
    ps.log2L = r[j] + rest;
    if (np == 1) ps.kind = SINGLE;
    else if (j == 0) ps.kind = FIRST;
    else if (j == np - 1) ps.kind = LAST;
    else ps.kind = MID;
    // the first pass of a large complex128 array reads rows 2^(e-R) elements
    // apart, each in its own page; wider tiles move twice the bytes per row
    // (complex64: 16384-element tiles, the first pass of 2^10 rows on the
    // radix-32 kernel and the middle pass of 2^11 rows)
    ps.wide = wide_on && (c128 ? ps.kind == FIRST && (r[j] == 10 || r[j] == 11)
                               : (ps.kind == FIRST && r[j] == 10) || (ps.kind == MID && r[j] == 11));
    int log2C = (ps.wide ? (c128 ? kLog2CtaWide : kLog2CtaWideC64) : log2cta) - r[j];
    if (log2C > e - r[j]) log2C = e - r[j];
    ps.log2C = log2C;
    ps.grid = 1ull << (e - r[j] - log2C);
    ps.threads = 1 << (r[j] + log2C - 4);
    const size_t elems = 1ull << (r[j] + log2C);
    ps.smem = (elems + elems / 16 + 1) * eb;
  }
  p->permute = (np >= 2) && !(p->flags & EFFT_FLAG_DIGIT_REVERSED_OUT);
  p->perm_log2A = (np >= 2) ? r[0] : 0;
  p->perm_B = (np == 3) ? (1u << r[1]) : 1u;
  // complex128 (a, b, a): the middle pass swaps the outer digits in place
  // (pairs of T x T column tiles held by the two CTAs of a cluster), so the
  // array reaches natural order without a separate swap sweep; the last pass
  // then transforms the columns of the swapped layout, strided like the
  // first pass, on 8192-element tiles.
  // The size rule folds only middle radices 2^8 and 2^10 (two CTAs per SM);
  // the 2^11 swapping pass (one 512-thread CTA per SM) is slower than the
  // swap sweep it saves at every size measured, and is reached only through
  // an explicit variant.
  const bool fuse_mid = (r[1] == 8 || r[1] == 10) || (v.fuse > 0 && r[1] == 11);
  if (fuse_on && p->permute && np == 3 && c128 && r[0] >= 9 && r[0] <= 11 && fuse_mid) {
    Pass& m = p->pass[1];
    m.swap = (r[1] == 8) ? 2 : 1;
    m.log2C = 2 * m.swap;
    m.wide = false;
    m.grid = 1ull << (e - r[1] - m.log2C);
    m.threads = 1 << (r[1] + m.log2C - 4);
    const size_t me = 1ull << (r[1] + m.log2C);
    m.smem = (me + me / 16 + 1) * eb;
    Pass& l = p->pass[2];
    l.kind = LASTS;
    l.log2s = e - r[2];
    l.log2L = e;
    l.wide = false;  // always on 8192-element tiles (not a variant of its own)
    l.log2C = kLog2CtaWide - r[2];
    l.grid = 1ull << (e - kLog2CtaWide);
    l.threads = 1 << (kLog2CtaWide - 4);
    const size_t le = 1ull << kLog2CtaWide;
    l.smem = (le + le / 16 + 1) * eb;
    p->permute = false;
  }
  // complex64: the wide first pass (2^10 rows, 16 columns) and the wide
  // middle pass (2^11 rows, 8 columns) fed by TMA copies
  if (!c128 && on(v.tma, kTmaRule)) {
    for (int j = 0; j < np; ++j) {
      Pass& f = p->pass[j];
      if (f.kind == FIRST) f.tma = f.wide && f.log2R == 10 && f.log2C == kLog2CtaWideC64 - 10;
      if (f.kind == MID) f.tma = f.wide && f.log2R == 11 && f.log2C == kLog2CtaWideC64 - 11 && f.log2s >= 3;
    }
  }
  // persistent prefetching kernels for the complex128 strided passes with a
  // tile shape they are built for.  The rule (measured, 2^28..2^33): they
  // pay for the one-CTA-per-SM passes -- the strided last pass at every
  // size, the wide first pass up to 2^31 (beyond, its burst of copies meets
  // address-translation misses) -- and not for the two-CTA-per-SM middle
  // passes or the swapping ones.
  if (c128 && pf != 0 && e >= kPersistMinLog2N) {
    for (int j = 0; j < np; ++j) {
      Pass& ps = p->pass[j];
      const int lr = ps.log2R, lc = ps.log2C;
      bool shape = false, rule = false;
      if (ps.swap) {
        shape = (lr == 11 && lc == 2) || (lr == 10 && lc == 2) || (lr == 8 && lc == 4);
      } else if (ps.kind == FIRST) {
        shape = ps.wide && ((lr == 10 && lc == 3) || (lr == 11 && lc == 2));
        rule = e <= kPersistFirstMaxLog2N;
      } else if (ps.kind == MID) {
        shape = (lr >= 8 && lr <= 11 && lr + lc == kLog2CtaC128);
      } else if (ps.kind == LASTS) {
        shape = (lr >= 9 && lr <= 11 && lr + lc == kLog2CtaWide);
        rule = true;
      }
      ps.pf = shape && (pf > 0 || rule);
    }
  }
}

Variant realised_variant(const efft_plan_s* p) {
  Variant v;
  v.wide = v.fuse = v.pf = v.tma = 0;
  for (int j = 0; j < p->npasses; ++j) {
    if (p->pass[j].wide) v.wide = 1;
    if (p->pass[j].swap) v.fuse = 1;
    if (p->pass[j].pf) v.pf = 1;
    if (p->pass[j].tma) v.tma = 1;
  }
  return v;
}

// cuTensorMapEncodeTiled through the runtime's driver entry-point query (no
// link-time libcuda); NULL when the driver does not offer it.
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiled encode_tiled() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
    cudaGetLastError();
  });
  return fn;
}

// The tensor map of a complex64 middle pass of R = 2^log2R rows at stride
// s = 2^log2s: the array as [N / (R s)][R][s] 8-byte elements, boxes of
// C x 256 x 1, no swizzle.
static bool mid_pass_map(CUtensorMap* map, void* data, int log2N, int log2R, int log2s, int C) {
  EncodeTiled fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(data) & 15u)) return false;
  const cuuint64_t dims[3] = {1ull << log2s, 1ull << log2R, 1ull << (log2N - log2R - log2s)};
  const cuuint64_t strides[2] = {(1ull << log2s) * 8, (1ull << (log2R + log2s)) * 8};
  const cuuint32_t box[3] = {(cuuint32_t)C, 256, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, data, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// The tensor map of a complex64 first pass of 2^10 rows: the array as
// [1024][s] 8-byte elements (s = N / 1024), 16 x 256 boxes, no swizzle.
static bool first_pass_map(CUtensorMap* map, void* data, int log2s) {
  EncodeTiled fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(data) & 15u)) return false;
  const cuuint64_t dims[2] = {1ull << log2s, 1024};
  const cuuint64_t strides[1] = {(1ull << log2s) * 8};
  const cuuint32_t box[2] = {16, 256};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, data, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <class P, int KIND, int CTA>
void set_smem_attr() {
  cudaFuncSetAttribute(efft_pass<P, KIND, CTA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((CTA + CTA / 16 + 1) * P::kElemBytes));
}

// The calling thread's current context: its device ordinal and the driver's
// context ID (unique for the life of the process, so a context destroyed and
// created again, e.g. after cudaDeviceReset, gets a new one).  The driver
// functions come through the runtime's entry-point query, so the library
// needs no link-time libcuda.  cudaSetDevice makes the device's primary
// context current (it creates it if there is none yet).
int current_context(int* dev, unsigned long long* ctx_id) {
  typedef int (*GetCurrent)(void**);
  typedef int (*GetId)(void*, unsigned long long*);
  static std::once_flag once;
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  if (cudaGetDevice(dev) != cudaSuccess || cudaSetDevice(*dev) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  *ctx_id = 0;
  void* ctx = nullptr;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx) {
    unsigned long long id = 0;
    if (get_id(ctx, &id) == 0) *ctx_id = id;
  }
  return EFFT_OK;
}

// Kernel attributes (the dynamic shared-memory limits) are set once per
// context: a context of another device, or a new context after a reset,
// gets them set again.  A failure is not remembered, so the next call
// retries.
int init_kernels() {
  constexpr int kSlots = 64;
  static std::mutex mu;
  static int done_dev[kSlots];
  static unsigned long long done_ctx[kSlots];
  static int ndone = 0;
  int dev = 0;
  unsigned long long ctx = 0;
  if (current_context(&dev, &ctx) != EFFT_OK) return EFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < ndone; ++i)
    if (done_dev[i] == dev && done_ctx[i] == ctx) return EFFT_OK;
  cudaGetLastError();  // a non-sticky error left by earlier calls is not ours
  {
    set_smem_attr<PolicyDF, FIRST, 1 << kLog2CtaC128>();
    set_smem_attr<PolicyDF, MID, 1 << kLog2CtaC128>();
    set_smem_attr<PolicyDF, LAST, 1 << kLog2CtaC128>();
    set_smem_attr<PolicyDF, SINGLE, 1 << kLog2CtaC128>();
    set_smem_attr<PolicyF32, FIRST, 1 << kLog2CtaC64>();
    set_smem_attr<PolicyF32, MID, 1 << kLog2CtaC64>();
    set_smem_attr<PolicyF32, LAST, 1 << kLog2CtaC64>();
    set_smem_attr<PolicyF32, SINGLE, 1 << kLog2CtaC64>();
    cudaError_t e0 = mix_set_attrs();
    cudaError_t e1 = fx_set_attrs_df2();
    cudaError_t e2 = fx_set_attrs_f32();
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = (e0 != cudaSuccess) ? e0 : (e1 != cudaSuccess) ? e1 : e2;
    if (err != cudaSuccess) return EFFT_ERR_CUDA;
  }
  // the table is small: when full, the oldest entry makes room
  if (ndone == kSlots) {
    for (int i = 1; i < kSlots; ++i) {
      done_dev[i - 1] = done_dev[i];
      done_ctx[i - 1] = done_ctx[i];
    }
    --ndone;
  }
  done_dev[ndone] = dev;
  done_ctx[ndone] = ctx;
  ++ndone;
  return EFFT_OK;
}

int gen_table(float4* out, uint64_t count, uint64_t stride, uint64_t N, cudaStream_t st) {
  const int bs = 256;
  uint64_t grid = (count + bs - 1) / bs;
  efft_twiddles<<<(unsigned)grid, bs, 0, st>>>(out, count, stride, N);
  return cudaGetLastError() == cudaSuccess ? EFFT_OK : EFFT_ERR_LAUNCH;
}

void release_events(efft_plan_s* p) {
  if (p->recs) {
    for (auto& r : *p->recs) {
      p->pool->push_back(r.a);
      p->pool->push_back(r.b);
    }
    p->recs->clear();
  }
}

void free_plan_memory(efft_plan_s* p) {
  if (p->recs) {
    release_events(p);
    delete p->recs;
    p->recs = nullptr;
  }
  if (p->pool) {
    for (cudaEvent_t e : *p->pool) cudaEventDestroy(e);
    delete p->pool;
    p->pool = nullptr;
  }
  if (p->ring) {
    for (int k = 0; k < kStateRing; ++k)
      if (p->ring->done[k]) {
        cudaEventSynchronize(p->ring->done[k]);
        cudaEventDestroy(p->ring->done[k]);
      }
    delete p->ring;
    p->ring = nullptr;
  }
  if (p->w2048) cudaFree(p->w2048);
  if (p->tw_lo) cudaFree(p->tw_lo);
  if (p->tw_hi) cudaFree(p->tw_hi);
  if (p->state) cudaFree(p->state);
  if (p->rtw_lo) cudaFree(p->rtw_lo);
  if (p->rtw_hi) cudaFree(p->rtw_hi);
  if (p->inner) efft_plan_destroy(p->inner);
  p->w2048 = p->tw_lo = p->tw_hi = p->rtw_lo = p->rtw_hi = nullptr;
  p->state = nullptr;
  p->inner = nullptr;
}

cudaEvent_t take_event(efft_plan_s* p) {
  cudaEvent_t e = nullptr;
  if (!p->pool->empty()) {
    e = p->pool->back();
    p->pool->pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records event a before a launch; returns the index of the record or -1.
int prof_begin(efft_plan_s* p, int slot, cudaStream_t st) {
  if (!p->profiling) return -1;
  cudaEvent_t a = take_event(p), b = take_event(p);
  if (!a || !b) return -1;
  cudaEventRecord(a, st);
  p->recs->push_back({slot, a, b});
  return (int)p->recs->size() - 1;
}
void prof_end(efft_plan_s* p, int rec, cudaStream_t st) {
  if (rec >= 0) cudaEventRecord((*p->recs)[rec].b, st);
}

// P: policy of the generic kernel; PFX: policy of the specialised kernels
template <class P, class PFX, int CTA>
cudaError_t launch_pass(const efft_plan_s* p, const Pass& ps, void* data, const Batch& bt, cudaStream_t st) {
  if (ps.mixed) return launch_mix(p, ps, data, bt, st);
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.log2R = ps.log2R;
  a.log2C = ps.log2C;
  a.log2s = ps.log2s;
  a.log2L = ps.log2L;
  a.log2N = p->log2n;
  a.twB = p->twB;
  a.w2048 = p->w2048;
  a.tw_lo = p->tw_lo;
  a.tw_hi = p->tw_hi;
  a.state = bt.state;
  a.ptrs = bt.ptrs;
  const uint32_t conj = (p->sign > 0) ? 1u : 0u;
  a.conj_in = (ps.kind == FIRST || ps.kind == SINGLE) ? conj : 0u;
  const bool last = (ps.kind == LAST || ps.kind == SINGLE || ps.kind == LASTS);
  a.conj_out = last ? conj : 0u;
  a.out_shift = ((p->flags & EFFT_FLAG_NORMALIZE) && last) ? p->log2n : 0;
  a.s_odd = (ps.kind == FIRST && p->odd > 1) ? p->odd : 1u;
  dim3 grid((unsigned)ps.grid, bt.count), block(ps.threads);
  constexpr int LOG2CTA = (P::kElemBytes == 16) ? kLog2CtaC128 : kLog2CtaC64;
  if (P::kElemBytes == 16 && ps.pf) {
    // persistent: at most as many CTAs (CTA pairs) as can be resident
    const int minb = (ps.log2R + ps.log2C == kLog2CtaWide) ? 1 : 2;
    const uint64_t cap = (uint64_t)(p->sms > 0 ? p->sms : 152) * minb;
    const uint64_t ntiles = ps.swap ? ps.grid / 2 : ps.grid;
    const uint64_t g = ps.swap ? 2 * std::min<uint64_t>(ntiles, cap / 2) : std::min<uint64_t>(ntiles, cap);
    a.ntiles = ntiles;
    const bool ok = fx_launch_df2_pf(ps.kind, ps.log2R, ps.log2C, ps.swap, dim3((unsigned)g, bt.count), block,
                                     ps.smem, st, data, a);
    return ok ? cudaGetLastError() : cudaErrorInvalidConfiguration;
  }
  if (P::kElemBytes == 16 && ps.swap) {
    const bool ok = fx_launch_df2_swap(ps.log2R, ps.log2C, grid, block, ps.smem, st, data, a);
    return ok ? cudaGetLastError() : cudaErrorInvalidConfiguration;
  }
  if (P::kElemBytes == 16 && ps.kind == LASTS) {
    const bool ok = fx_launch_df2_lasts(ps.log2R, grid, block, ps.smem, st, data, a);
    return ok ? cudaGetLastError() : cudaErrorInvalidConfiguration;
  }
  if (P::kElemBytes == 8 && ps.tma && !bt.ptrs) {
    CUtensorMap map;
    const bool first = (ps.kind == FIRST);
    if (first ? first_pass_map(&map, data, ps.log2s)
              : mid_pass_map(&map, data, p->log2n, ps.log2R, ps.log2s, 1 << ps.log2C)) {
      // (word 3 of the state, this execute's record of an expired device
      // wait, was cleared by enqueue_batch)
      a.ntiles = ps.grid;
      a.inject_timeout = fault_injected("tma_wait") ? 1u : 0u;
      const uint64_t g = std::min<uint64_t>(ps.grid, (uint64_t)(p->sms > 0 ? p->sms : 152));
      const bool ok = first ? fx_launch_f32_tma(dim3((unsigned)g, 1), st, data, a, &map)
                            : fx_launch_f32_mid_tma(dim3((unsigned)g, 1), st, data, a, &map);
      return ok ? cudaGetLastError() : cudaErrorInvalidConfiguration;
    }
    // no tensor map (no driver entry point, or a buffer not 16-byte
    // aligned): the same pass on the kernel that loads its own tiles
  }
  if (ps.wide) {
    const bool ok = (P::kElemBytes == 16) ? fx_launch_df2_wide(ps.log2R, grid, block, ps.smem, st, data, a)
                                          : fx_launch_f32_wide(ps.kind, ps.log2R, grid, st, data, a);
    return ok ? cudaGetLastError() : cudaErrorInvalidConfiguration;
  }
  if (ps.kind != SINGLE && ps.log2R >= 8 && ps.log2R <= 11 && ps.log2R + ps.log2C == LOG2CTA) {
    const bool ok = (P::kElemBytes == 16) ? fx_launch_df2(ps.kind, ps.log2R, grid, block, ps.smem, st, data, a)
                                          : fx_launch_f32(ps.kind, ps.log2R, grid, block, ps.smem, st, data, a);
    if (ok) return cudaGetLastError();
  }
  if (p->odd > 1) return cudaErrorInvalidConfiguration;  // only the specialised kernels take s_odd
  switch (ps.kind) {
    case FIRST: efft_pass<P, FIRST, CTA><<<grid, block, ps.smem, st>>>(data, a); break;
    case MID: efft_pass<P, MID, CTA><<<grid, block, ps.smem, st>>>(data, a); break;
    case LAST: efft_pass<P, LAST, CTA><<<grid, block, ps.smem, st>>>(data, a); break;
    default: efft_pass<P, SINGLE, CTA><<<grid, block, ps.smem, st>>>(data, a); break;
  }
  return cudaGetLastError();
}

}  // namespace host
}  // namespace efft

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int efft_version(void) { return EFFT_VERSION; }

const char* efft_strerror(int s) {
  switch (s) {
    case EFFT_OK: return "success";
    case EFFT_ERR_INVALID_SIZE: return "invalid size: N must be 2^e with 0 <= e <= 33";
    case EFFT_ERR_INVALID_DTYPE: return "invalid dtype: expected EFFT_C64 or EFFT_C128";
    case EFFT_ERR_INVALID_SIGN: return "invalid sign: expected -1 or +1";
    case EFFT_ERR_INVALID_PTR: return "invalid pointer: NULL or not device memory of the plan's device";
    case EFFT_ERR_MISALIGNED: return "misaligned pointer: must be aligned to the element size";
    case EFFT_ERR_ALLOC: return "allocation failed";
    case EFFT_ERR_LAUNCH: return "kernel launch or copy rejected";
    case EFFT_ERR_TIMEOUT: return "a bounded device wait expired";
    case EFFT_ERR_UNSUPPORTED: return "unsupported request";
    case EFFT_ERR_INVALID_PLAN: return "invalid plan handle (NULL, destroyed or foreign)";
    case EFFT_ERR_CUDA: return "CUDA runtime error (no device or bad context)";
    case EFFT_ERR_INVALID_FLAGS: return "unknown flag bits";
    default: return "unknown status";
  }
}

}  // extern "C"

namespace efft {
namespace host {

// Plan creation; r_explicit != NULL: the caller's schedule (already checked).
int plan_create_impl(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags, const int* r_explicit,
                     int np_explicit) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  if (init_kernels() != EFFT_OK) return EFFT_ERR_CUDA;

  efft_plan_s* p = new (std::nothrow) efft_plan_s();
  if (!p) return EFFT_ERR_ALLOC;
  std::memset(p, 0, sizeof(*p));
  p->device = dev;
  p->n = n;
  p->log2n = ilog2_u64(n);
  p->dtype = dtype;
  p->sign = sign;
  p->flags = flags;
  if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    p->sms = 0;
  }

  const int e = p->log2n;  // ceil(log2 N)
  const size_t eb = (dtype == EFFT_C128) ? 16 : 8;
  p->odd = (uint32_t)(n / (n & (~n + 1)));
  bool tune = false;
  Tuned t;
  const bool cached = (flags & EFFT_FLAG_AUTOTUNE) && !r_explicit && tuned_lookup(dev, n, dtype, &t);
  if (p->odd > 1) {
    // N = M * 2^e: the mixed-radix schedule (the tuned outer radix if cached)
    const int force = r_explicit ? (np_explicit == 3 ? r_explicit[0] : 0) : (cached ? t.mixed_a : -1);
    const int rc0 = apply_mixed_schedule(p, force, (cached && !r_explicit) ? t.v : Variant());
    if (rc0 != EFFT_OK) {
      delete p;
      return rc0;
    }
    tune = (flags & EFFT_FLAG_AUTOTUNE) && !cached && n > 2048 && n * eb <= EFFT_AUTOTUNE_MAX_BYTES;
  } else if (r_explicit) {
    apply_schedule(p, r_explicit, np_explicit);
  } else if (cached) {
    apply_schedule(p, t.r, t.np, t.v);
  } else {
    int r[kMaxPasses] = {0, 0, 0, 0};
    const int np = choose_radices(e, r);
    apply_schedule(p, r, np);
    tune = (flags & EFFT_FLAG_AUTOTUNE) && e >= 4 && n * eb <= EFFT_AUTOTUNE_MAX_BYTES;
  }
  p->twB = (e + 1) / 2;

  if (fault_injected("alloc")) {
    delete p;
    return EFFT_ERR_ALLOC;
  }
  const uint64_t nlo = 1ull << p->twB, nhi = (n + nlo - 1) >> p->twB;
  cudaStream_t st = nullptr;
  int rc = EFFT_OK;
  if (cudaMalloc(&p->w2048, 2048 * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&p->tw_lo, nlo * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&p->tw_hi, nhi * sizeof(float4)) != cudaSuccess) {
    rc = EFFT_ERR_ALLOC;
  }
  if (rc == EFFT_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = EFFT_ERR_CUDA;
  if (rc == EFFT_OK) rc = gen_table(p->w2048, 2048, 1, 2048, st);
  if (rc == EFFT_OK) rc = gen_table(p->tw_lo, nlo, 1, n, st);
  if (rc == EFFT_OK) rc = gen_table(p->tw_hi, nhi, nlo, n, st);
  if (rc == EFFT_OK) rc = ring_create(p, st);
  if (rc == EFFT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = EFFT_ERR_CUDA;
  p->recs = new (std::nothrow) std::vector<efft_plan_s::Rec>();
  p->pool = new (std::nothrow) std::vector<cudaEvent_t>();
  if (rc == EFFT_OK && (!p->recs || !p->pool)) rc = EFFT_ERR_ALLOC;
  if (rc == EFFT_OK && tune) {
    // a temporary buffer; without room the table's schedule stays
    void* scratch = nullptr;
    if (cudaMalloc(&scratch, n * eb) == cudaSuccess) {
      rc = autotune_impl(p, scratch, st, nullptr, 0, nullptr);
      cudaFree(scratch);
    } else {
      cudaGetLastError();
    }
  }
  if (st) cudaStreamDestroy(st);
  if (rc != EFFT_OK) {
    cudaGetLastError();
    free_plan_memory(p);
    delete p;
    return rc;
  }
  p->table_bytes = (2048 + nlo + nhi) * sizeof(float4) + 16 * kStateRing;
  p->magic = kMagic;
  register_plan(p);
  *out = p;
  return EFFT_OK;
}

int check_create_args(efft_plan_t* out, uint64_t n, int dtype, int sign) {
  if (!out) return EFFT_ERR_INVALID_PTR;
  *out = nullptr;
  if (!valid_size(n)) return EFFT_ERR_INVALID_SIZE;
  if (dtype != EFFT_C64 && dtype != EFFT_C128) return EFFT_ERR_INVALID_DTYPE;
  if (sign != -1 && sign != 1) return EFFT_ERR_INVALID_SIGN;
  return EFFT_OK;
}

}  // namespace host
}  // namespace efft

extern "C" {

int efft_plan_create(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags) {
  int rc = check_create_args(out, n, dtype, sign);
  if (rc != EFFT_OK) return rc;
  if (flags & ~EFFT_FLAG_ALL) return EFFT_ERR_INVALID_FLAGS;
  // 1/N is exact in binary floating point only for N a power of two
  if ((n & (n - 1)) != 0 && (flags & EFFT_FLAG_NORMALIZE)) return EFFT_ERR_UNSUPPORTED;
  return plan_create_impl(out, n, dtype, sign, flags, nullptr, 0);
}

int efft_plan_create_with_radices(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags,
                                  const int* log2_radices, int npasses) {
  int rc = check_create_args(out, n, dtype, sign);
  if (rc != EFFT_OK) return rc;
  if (flags & ~(EFFT_FLAG_ALL & ~EFFT_FLAG_AUTOTUNE)) return EFFT_ERR_INVALID_FLAGS;
  if ((n & (n - 1)) != 0) {
    if (!valid_mixed_schedule(n, dtype, log2_radices, npasses)) return EFFT_ERR_UNSUPPORTED;
  } else if (!valid_schedule(ilog2_u64(n), log2_radices, npasses)) {
    return EFFT_ERR_UNSUPPORTED;
  }
  static const int kNone[1] = {0};
  return plan_create_impl(out, n, dtype, sign, flags, log2_radices ? log2_radices : kNone, npasses);
}

int efft_plan_destroy(efft_plan_t plan) {
  if (!plan) return EFFT_OK;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_live || !g_live->count(plan) || plan->magic != kMagic) return EFFT_ERR_INVALID_PLAN;
    g_live->erase(plan);
  }
  plan->magic = 0;
  {
    DeviceGuard g(plan->device);
    free_plan_memory(plan);
  }
  delete plan;
  return EFFT_OK;
}

int efft_plan_radices(efft_plan_t plan, int* log2_radices, int cap, int* npasses) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (plan->real) plan = plan->inner;  // the complex plan of n/2 points
  if (npasses) *npasses = plan->npasses;
  if (log2_radices)
    for (int j = 0; j < plan->npasses && j < cap; ++j) log2_radices[j] = plan->pass[j].log2R;
  return EFFT_OK;
}

int efft_plan_schedule(uint64_t n, int dtype, uint64_t* radices, int cap, int* npasses) {
  if (!npasses) return EFFT_ERR_INVALID_PTR;
  if (!valid_size(n)) return EFFT_ERR_INVALID_SIZE;
  if (dtype != EFFT_C64 && dtype != EFFT_C128) return EFFT_ERR_INVALID_DTYPE;
  efft_plan_s p;
  std::memset(&p, 0, sizeof(p));
  p.n = n;
  p.log2n = ilog2_u64(n);
  p.dtype = dtype;
  p.odd = (uint32_t)(n / (n & (~n + 1)));
  if (p.odd > 1) {
    const int rc = apply_mixed_schedule(&p);
    if (rc != EFFT_OK) return rc;
  } else {
    int r[kMaxPasses] = {0, 0, 0, 0};
    apply_schedule(&p, r, choose_radices(p.log2n, r));
  }
  *npasses = p.npasses;
  for (int j = 0; radices && j < p.npasses && j < cap; ++j)
    radices[j] = (p.odd > 1) ? p.pass[j].R_int : (1ull << p.pass[j].log2R);
  return EFFT_OK;
}

int efft_plan_info(efft_plan_t plan, double* hbm_passes, uint64_t* table_bytes) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (plan->real) {
    // the complex plan's sweeps of the same bytes, the mirrored-pair sweep,
    // and for an inverse complex128 plan the range scan ahead of it
    double hp = 0.0;
    uint64_t tb = 0;
    efft_plan_info(plan->inner, &hp, &tb);
    if (hbm_passes) *hbm_passes = hp + 1.0 + ((plan->dtype == EFFT_C128 && plan->real > 0) ? 0.5 : 0.0);
    if (table_bytes) *table_bytes = tb + plan->table_bytes;
    return EFFT_OK;
  }
  if (hbm_passes) {
    double hp = plan->npasses + (plan->permute ? 1.0 : 0.0);
    if (plan->small) hp = 1.0;
    if (plan->dtype == EFFT_C128 && plan->log2n > 0) hp += 0.5;
    *hbm_passes = hp;
  }
  if (table_bytes) *table_bytes = plan->table_bytes;
  return EFFT_OK;
}

}  // extern "C"

namespace efft {
namespace host {

size_t plan_bytes(const efft_plan_s* p) {
  const size_t s = (p->dtype == EFFT_C128) ? 16 : 8;
  return p->n * (p->real ? s / 2 : s);
}

// Clears the state words and enqueues the range scan of `count` arrays of
// n_complex complex128 values (data, or ptrs[0..count) when ptrs != NULL).
int launch_range_scan(const void* data, uint64_t n_complex, uint32_t* state, void* const* ptrs, unsigned count,
                      cudaStream_t st) {
  if (cudaMemsetAsync(state, 0, 16 * (size_t)count, st) != cudaSuccess) return EFFT_ERR_LAUNCH;
  uint64_t blocks = (n_complex + 1023) / 1024;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (ptrs && blocks * count > 152 * 16) blocks = (152 * 16 + count - 1) / count;
  efft_range_scan<<<dim3((unsigned)blocks, count), 256, 0, st>>>(reinterpret_cast<const uint4*>(data), n_complex,
                                                                 state, ptrs);
  return cudaGetLastError() == cudaSuccess ? EFFT_OK : EFFT_ERR_LAUNCH;
}

int check_buffer(const efft_plan_s* p, const void* data) {
  if (!data) return EFFT_ERR_INVALID_PTR;
  const uintptr_t align = (p->dtype == EFFT_C128) ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(data) % align) return EFFT_ERR_MISALIGNED;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, data) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_INVALID_PTR;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return EFFT_ERR_INVALID_PTR;
  if (attr.device != p->device) return EFFT_ERR_INVALID_PTR;
  return EFFT_OK;
}

// One transform at `data`, or bt.count transforms (bt.ptrs) of the plan's
// size in the same launches.
int enqueue_batch(efft_plan_s* p, void* data, const Batch& bt, cudaStream_t st) {
  if (fault_injected("launch")) return EFFT_ERR_LAUNCH;
  if (p->log2n == 0 || bt.count == 0) return EFFT_OK;  // N = 1: the DFT is the identity
  const bool c128 = (p->dtype == EFFT_C128);
  if (c128) {
    int rec = prof_begin(p, 0, st);
    const int rc = launch_range_scan(data, p->n, bt.state, bt.ptrs, bt.count, st);
    prof_end(p, rec, st);
    if (rc != EFFT_OK) return rc;
  }
  if (p->small) {
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.log2N = p->log2n;
    a.w2048 = p->w2048;
    a.state = bt.state;
    a.ptrs = bt.ptrs;
    a.conj_in = a.conj_out = (p->sign > 0) ? 1u : 0u;
    a.out_shift = (p->flags & EFFT_FLAG_NORMALIZE) ? p->log2n : 0;
    int rec = prof_begin(p, 6, st);
    if (c128) efft_small<PolicyDF><<<dim3(1, bt.count), 32, 0, st>>>(data, a);
    else efft_small<PolicyF32><<<dim3(1, bt.count), 32, 0, st>>>(data, a);
    prof_end(p, rec, st);
    return cudaGetLastError() == cudaSuccess ? EFFT_OK : EFFT_ERR_LAUNCH;
  }
  // complex64 passes fed by TMA record an expired wait in word 3 of the
  // execute's state: cleared once per execute (complex128 executes clear
  // the whole word in the range scan)
  if (!c128 && !bt.ptrs) {
    bool tma = false;
    for (int j = 0; j < p->npasses; ++j) tma = tma || p->pass[j].tma;
    if (tma && cudaMemsetAsync(bt.state + 3, 0, 4, st) != cudaSuccess) return EFFT_ERR_LAUNCH;
  }
  for (int j = 0; j < p->npasses; ++j) {
    int rec = prof_begin(p, 1 + j, st);
    cudaError_t err = c128 ? launch_pass<PolicyDF, PolicyDF2, 1 << kLog2CtaC128>(p, p->pass[j], data, bt, st)
                           : launch_pass<PolicyF32, PolicyF32, 1 << kLog2CtaC64>(p, p->pass[j], data, bt, st);
    prof_end(p, rec, st);
    if (err != cudaSuccess) return EFFT_ERR_LAUNCH;
  }
  if (p->permute) {
    const int la = p->perm_log2A;
    const uint32_t B = p->perm_B;
    const int lt = la < 5 ? la : 5;
    const uint64_t nt = 1ull << (la - lt);
    dim3 grid((unsigned)(nt * (nt + 1) / 2), B, bt.count);
    int rec = prof_begin(p, 5, st);
    if (c128)
      efft_digit_swap<uint4><<<grid, 256, 0, st>>>(reinterpret_cast<uint4*>(data), la, B, lt,
                                                    reinterpret_cast<uint4* const*>(bt.ptrs));
    else
      efft_digit_swap<uint2><<<grid, 256, 0, st>>>(reinterpret_cast<uint2*>(data), la, B, lt,
                                                    reinterpret_cast<uint2* const*>(bt.ptrs));
    prof_end(p, rec, st);
    if (cudaGetLastError() != cudaSuccess) return EFFT_ERR_LAUNCH;
  }
  return EFFT_OK;
}

int enqueue_state(efft_plan_s* p, void* data, uint32_t* state, cudaStream_t st) {
  if (p->real) return enqueue_real(p, data, state, st);
  const Batch one{nullptr, 1u, state};
  return enqueue_batch(p, data, one, st);
}

int ring_create(efft_plan_s* p, cudaStream_t st) {
  p->ring = new (std::nothrow) StateRing();
  if (!p->ring) return EFFT_ERR_ALLOC;
  if (cudaMalloc(&p->state, 16 * (size_t)kStateRing) != cudaSuccess) return EFFT_ERR_ALLOC;
  for (int k = 0; k < kStateRing; ++k)
    if (cudaEventCreateWithFlags(&p->ring->done[k], cudaEventDisableTiming) != cudaSuccess) return EFFT_ERR_CUDA;
  return cudaMemsetAsync(p->state, 0, 16 * (size_t)kStateRing, st) == cudaSuccess ? EFFT_OK : EFFT_ERR_CUDA;
}

// Every execute has a state word of its own, so executes of one plan on
// different buffers may overlap.  Eager executes take the ring's next word,
// first waiting (on the device) for the execute that used it before.  An
// execute captured into a CUDA graph gets a word allocated in the graph by
// the stream-ordered allocator (an allocation node and a free node around
// its launches), so every launch of the graph has its own word and the ring
// is not touched by replays.
int enqueue(efft_plan_s* p, void* data, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  if (cs == cudaStreamCaptureStatusInvalidated) return EFFT_ERR_CUDA;
  if (cs == cudaStreamCaptureStatusActive) {
    void* word = nullptr;
    if (cudaMallocAsync(&word, 16, st) != cudaSuccess) {
      cudaGetLastError();
      return EFFT_ERR_ALLOC;
    }
    int rc = enqueue_state(p, data, static_cast<uint32_t*>(word), st);
    if (cudaFreeAsync(word, st) != cudaSuccess && rc == EFFT_OK) rc = EFFT_ERR_CUDA;
    return rc;
  }
  StateRing& r = *p->ring;
  std::lock_guard<std::mutex> lk(r.mu);
  const int k = r.next;
  if (r.used[k] && cudaStreamWaitEvent(st, r.done[k], 0) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  int rc = enqueue_state(p, data, p->state + 4 * k, st);
  // recorded even after a failed enqueue: the launches already made are
  // behind it
  if (cudaEventRecord(r.done[k], st) != cudaSuccess) {
    cudaGetLastError();
    if (rc == EFFT_OK) rc = EFFT_ERR_CUDA;
  } else {
    r.used[k] = true;
  }
  r.next = (k + 1) % kStateRing;
  return rc;
}

}  // namespace host
}  // namespace efft

extern "C" {

int efft_execute(efft_plan_t plan, void* data, void* stream) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  DeviceGuard g(plan->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  int rc = check_buffer(plan, data);
  if (rc != EFFT_OK) return rc;
  return enqueue(plan, data, reinterpret_cast<cudaStream_t>(stream));
}

int efft_execute_host(efft_plan_t plan, void* host_data, void* dev_data, void* stream) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (!host_data) return EFFT_ERR_INVALID_PTR;
  DeviceGuard g(plan->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  int rc = check_buffer(plan, dev_data);
  if (rc != EFFT_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = plan_bytes(plan);
  if (cudaMemcpyAsync(dev_data, host_data, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  rc = enqueue(plan, dev_data, st);
  if (rc != EFFT_OK) return rc;
  if (cudaMemcpyAsync(host_data, dev_data, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  return EFFT_OK;
}

int efft_execute_host_stream(const efft_plan_t* plans, int nplans, void* const* host_in,
                             void* const* host_out, int count, void* const* dev_bufs, int nbufs,
                             void* stream) {
  if (!plans || nplans < 1 || nbufs < 1 || count < 0) return EFFT_ERR_INVALID_SIZE;
  for (int j = 0; j < nplans; ++j) {
    if (!plan_is_live(plans[j])) return EFFT_ERR_INVALID_PLAN;
    if (plan_bytes(plans[j]) != plan_bytes(plans[0]) || plans[j]->dtype != plans[0]->dtype ||
        plans[j]->device != plans[0]->device)
      return EFFT_ERR_INVALID_SIZE;
  }
  if (count == 0) return EFFT_OK;
  if (!host_in || !host_out || !dev_bufs) return EFFT_ERR_INVALID_PTR;
  for (int i = 0; i < count; ++i)
    if (!host_in[i] || !host_out[i]) return EFFT_ERR_INVALID_PTR;
  efft_plan_s* p0 = plans[0];
  DeviceGuard g(p0->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  for (int b = 0; b < nbufs; ++b) {
    int rc = check_buffer(p0, dev_bufs[b]);
    if (rc != EFFT_OK) return rc;
  }
  const size_t bytes = plan_bytes(p0);
  cudaStream_t sc = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t sin = nullptr, sout = nullptr;
  // one copy-out event per 1 GiB piece of each buffer: the next array's copy
  // of a piece into the buffer waits only for that piece's copy out, so with
  // one buffer the copy out of array i and the copy in of array i+1 share the
  // link's two directions
  const size_t npieces = (bytes + kCopyChunk - 1) / kCopyChunk;
  std::vector<cudaEvent_t> ev_in(nbufs, nullptr), ev_comp(nbufs, nullptr), ev_out(nbufs * npieces, nullptr);
  std::vector<bool> used(nbufs, false);
  int rc = EFFT_OK;
  if (cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking) != cudaSuccess)
    rc = EFFT_ERR_CUDA;
  for (int b = 0; rc == EFFT_OK && b < nbufs; ++b) {
    if (cudaEventCreateWithFlags(&ev_in[b], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_comp[b], cudaEventDisableTiming) != cudaSuccess)
      rc = EFFT_ERR_CUDA;
    for (size_t q = 0; rc == EFFT_OK && q < npieces; ++q)
      if (cudaEventCreateWithFlags(&ev_out[b * npieces + q], cudaEventDisableTiming) != cudaSuccess)
        rc = EFFT_ERR_CUDA;
  }
  for (int i = 0; rc == EFFT_OK && i < count; ++i) {
    const int b = i % nbufs;
    void* buf = dev_bufs[b];
    // copies in 1 GiB pieces: the two copy directions then interleave on the
    // link (measured 16+16 GiB: 118 ms whole, 100 ms in pieces); each piece
    // once the buffer's previous result has left that piece
    for (size_t o = 0, q = 0; rc == EFFT_OK && o < bytes; o += kCopyChunk, ++q) {
      const size_t len = (bytes - o < kCopyChunk) ? bytes - o : kCopyChunk;
      if (used[b] && cudaStreamWaitEvent(sin, ev_out[b * npieces + q], 0) != cudaSuccess) rc = EFFT_ERR_CUDA;
      else if (cudaMemcpyAsync(static_cast<char*>(buf) + o, static_cast<const char*>(host_in[i]) + o, len,
                               cudaMemcpyHostToDevice, sin) != cudaSuccess)
        rc = EFFT_ERR_CUDA;
    }
    if (rc != EFFT_OK || cudaEventRecord(ev_in[b], sin) != cudaSuccess) { rc = EFFT_ERR_CUDA; break; }
    // transforms in order on the caller's stream
    if (cudaStreamWaitEvent(sc, ev_in[b], 0) != cudaSuccess) { rc = EFFT_ERR_CUDA; break; }
    for (int j = 0; rc == EFFT_OK && j < nplans; ++j) rc = enqueue(plans[j], buf, sc);
    if (rc != EFFT_OK) break;
    if (cudaEventRecord(ev_comp[b], sc) != cudaSuccess) { rc = EFFT_ERR_CUDA; break; }
    // copy out
    if (cudaStreamWaitEvent(sout, ev_comp[b], 0) != cudaSuccess) { rc = EFFT_ERR_CUDA; break; }
    for (size_t o = 0, q = 0; rc == EFFT_OK && o < bytes; o += kCopyChunk, ++q) {
      const size_t len = (bytes - o < kCopyChunk) ? bytes - o : kCopyChunk;
      if (cudaMemcpyAsync(static_cast<char*>(host_out[i]) + o, static_cast<const char*>(buf) + o, len,
                          cudaMemcpyDeviceToHost, sout) != cudaSuccess ||
          cudaEventRecord(ev_out[b * npieces + q], sout) != cudaSuccess)
        rc = EFFT_ERR_CUDA;
    }
    if (rc != EFFT_OK) break;
    used[b] = true;
  }
  // drain everything that was enqueued, even after an error
  if (sin) cudaStreamSynchronize(sin);
  cudaStreamSynchronize(sc);
  if (sout && cudaStreamSynchronize(sout) != cudaSuccess && rc == EFFT_OK) rc = EFFT_ERR_CUDA;
  for (int b = 0; b < nbufs; ++b) {
    if (ev_in[b]) cudaEventDestroy(ev_in[b]);
    if (ev_comp[b]) cudaEventDestroy(ev_comp[b]);
  }
  for (cudaEvent_t e : ev_out)
    if (e) cudaEventDestroy(e);
  if (sin) cudaStreamDestroy(sin);
  if (sout) cudaStreamDestroy(sout);
  if (rc != EFFT_OK) cudaGetLastError();
  return rc;
}

int efft_execute_check(efft_plan_t plan, void* stream) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (plan->real) plan = plan->inner;
  DeviceGuard g(plan->device);
  if (!g.ok) return EFFT_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  if (plan->dtype != EFFT_C64) return EFFT_OK;  // complex128 kernels have no device waits
  uint32_t words[4 * kStateRing];
  if (cudaMemcpy(words, plan->state, sizeof(words), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  int rc = EFFT_OK;
  for (int k = 0; k < kStateRing; ++k)
    if (words[4 * k + 3] == (uint32_t)EFFT_ERR_TIMEOUT) rc = EFFT_ERR_TIMEOUT;
  if (rc != EFFT_OK && cudaMemset(plan->state, 0, sizeof(words)) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  return rc;
}

int efft_plan_profile(efft_plan_t plan, int enable) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  if (plan->real) efft_plan_profile(plan->inner, enable);
  DeviceGuard g(plan->device);
  if (enable) {
    for (auto& r : *plan->recs) cudaEventSynchronize(r.b);
    release_events(plan);
  }
  plan->profiling = enable != 0;
  return EFFT_OK;
}

int efft_plan_profile_read(efft_plan_t plan, double* ms, int* count, int cap, int* nslots) {
  if (!plan_is_live(plan)) return EFFT_ERR_INVALID_PLAN;
  DeviceGuard g(plan->device);
  double tot[EFFT_PROFILE_SLOTS] = {0};
  int cnt[EFFT_PROFILE_SLOTS] = {0};
  int rc = EFFT_OK;
  if (plan->real) {  // the complex plan's launches, then this plan's own
    double ims[EFFT_PROFILE_SLOTS] = {0};
    int icnt[EFFT_PROFILE_SLOTS] = {0};
    rc = efft_plan_profile_read(plan->inner, ims, icnt, EFFT_PROFILE_SLOTS, nullptr);
    for (int s = 0; s < EFFT_PROFILE_SLOTS; ++s) {
      tot[s] += ims[s];
      cnt[s] += icnt[s];
    }
  }
  for (auto& r : *plan->recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      rc = EFFT_ERR_CUDA;
      continue;
    }
    if (r.slot >= 0 && r.slot < EFFT_PROFILE_SLOTS) {
      tot[r.slot] += t;
      cnt[r.slot] += 1;
    }
  }
  release_events(plan);
  for (int s = 0; s < cap && s < EFFT_PROFILE_SLOTS; ++s) {
    if (ms) ms[s] = tot[s];
    if (count) count[s] = cnt[s];
  }
  if (nslots) *nslots = EFFT_PROFILE_SLOTS;
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal helper for efft_execute_noalloc (efft_noalloc.cu): the same launch
// sequence as efft_execute, for a plan description built on the stack whose
// twiddle tables and state word live in caller-provided device memory.
// Allocates nothing; enqueues the table generation first when `regen`.
// ---------------------------------------------------------------------------
int efft_internal_run_in_scratch(void* scratch, size_t scratch_bytes, bool regen, void* data, uint64_t n,
                                 int dtype, int sign, uint32_t flags, cudaStream_t st) {
  if (init_kernels() != EFFT_OK) return EFFT_ERR_CUDA;
  efft_plan_s p;
  std::memset(&p, 0, sizeof(p));
  if (cudaGetDevice(&p.device) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  p.n = n;
  p.log2n = ilog2_u64(n);
  p.dtype = dtype;
  p.sign = sign;
  p.flags = flags;
  p.odd = 1;  // powers of two only
  const int e = p.log2n;
  int r[kMaxPasses] = {0, 0, 0, 0};
  apply_schedule(&p, r, choose_radices(e, r));
  p.twB = (e + 1) / 2;
  const uint64_t nlo = 1ull << p.twB, nhi = 1ull << (e - p.twB);
  const size_t state_off = (2048 + nlo + nhi) * sizeof(float4);
  if (state_off + 16 > scratch_bytes) return EFFT_ERR_INVALID_SIZE;
  float4* base = reinterpret_cast<float4*>(scratch);
  p.w2048 = base;
  p.tw_lo = base + 2048;
  p.tw_hi = base + 2048 + nlo;
  p.state = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(scratch) + state_off);
  int rc = check_buffer(&p, data);
  if (rc != EFFT_OK) return rc;
  if (regen) {
    if ((rc = gen_table(p.w2048, 2048, 1, 2048, st)) != EFFT_OK) return rc;
    if ((rc = gen_table(p.tw_lo, nlo, 1, n, st)) != EFFT_OK) return rc;
    if ((rc = gen_table(p.tw_hi, nhi, nlo, n, st)) != EFFT_OK) return rc;
  }
  return enqueue_state(&p, data, p.state, st);
}
