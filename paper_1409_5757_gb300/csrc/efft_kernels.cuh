// efft_kernels.cuh -- device kernels of the in-place multi-pass DFT.
//
//   efft_pass       one in-place pass: a batch of strided size-R sub-DFTs in
//                   shared memory (Sec. 3.3 "processing"), radix-16 DIF
//                   stages, twiddles of Eq. 4 fused into the epilogue
//                   (Sec. 3.4 "reassembly"); results written back to the
//                   slots that were read (the in-place principle of Sec. 3.4).
//   efft_small      N <= 8: one thread evaluates Eq. 1 directly.
// The range scan (largest binary64 exponent of the input), the digit swap
// (digit-reversed pass output to natural order) and the twiddle-table
// kernel are in efft.cu with their launches.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "efft_arith.cuh"

namespace efft {

// Pass kinds for complex128 (double-float intermediate kept in the buffer):
//   FIRST  binary64 in  -> df out      MID  df in -> df out
//   LAST   df in        -> binary64    SINGLE binary64 in -> binary64 out
//   LASTS  df in        -> binary64, the last pass of a three-pass schedule
//          whose middle pass already swapped the outer digits: its columns
//          are strided like the first pass's (stride N / R), no twiddle.
enum PassKind { FIRST = 0, MID = 1, LAST = 2, SINGLE = 3, LASTS = 4 };

struct PassArgs {
  int log2R;        // radix of this pass, 4 <= log2R <= 11
  int log2C;        // columns per CTA: C = CTA_ELEMS / R
  int log2s;        // element stride inside a column (s = 1 for the last pass)
  int log2L;        // block length L = R * s
  int log2N;        // transform length
  int twB;          // low-table bits of the two-level twiddle table
  const float4* w2048;   // exp(-2*pi*i*t/2048), t < 2048
  const float4* tw_lo;   // exp(-2*pi*i*t/N), t < 2^twB
  const float4* tw_hi;   // exp(-2*pi*i*(t << twB)/N), t < N >> twB
  const uint32_t* state; // state[0] = max biased binary64 exponent of the input
  void* const* ptrs;     // non-null: batched launch, transform blockIdx.y has data
                         // ptrs[blockIdx.y] and state word state + 4*blockIdx.y
  uint32_t conj_in;      // 1: conjugate the input (sign = +1 transforms)
  uint32_t conj_out;     // 1: conjugate the output
  int out_shift;         // output multiplied by 2^-out_shift (1/N normalisation)
  uint32_t s_odd;        // first pass of N = M * 2^e: stride s = s_odd * 2^log2s
                         // (s_odd = M); 1 for power-of-two N
  uint64_t ntiles;       // persistent kernels: tiles per transform (a swapping
                         // pass: tile pairs)
  uint32_t inject_timeout;  // host-side fault injection: a TMA pass arms its
                            // barrier without copies (its bounded wait expires)
};

// Shared-memory slot of (position p, column c): one pad slot per 16 keeps the
// stride-16 accesses of the last stage free of bank conflicts.
__device__ __forceinline__ int smem_slot(int p, int c, int log2C) {
  int raw = (p << log2C) + c;
  return raw + (raw >> 4);
}

// ----------------------------------------------------------------------------
// binary64 <-> double-float conversion by integer bit manipulation.
// The array's values are scaled by 2^-(emax-1023), emax = the largest biased
// exponent in the input, so that the largest input has magnitude in [1, 2).
// D = emax - 127 is the exponent offset between a float and a binary64
// exponent field.
// ----------------------------------------------------------------------------
__device__ __forceinline__ df f64bits_to_df(uint32_t lo, uint32_t hi, int D, uint32_t flip) {
  uint32_t sign = (hi ^ flip) & 0x80000000u;
  int E = (int)((hi >> 20) & 0x7FFu);
  int fe = E - D;  // biased float exponent of the scaled value
  // high float: implicit 1 + top 23 of the 52 mantissa bits (truncated)
  uint32_t mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
  uint32_t hbits = sign | ((uint32_t)fe << 23) | mant;
  // low float: the remaining 29 mantissa bits rounded to 24, times
  // 2^(fe - 127 - 52) (an exact power-of-two scaling)
  float l = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), __uint_as_float((uint32_t)(fe - 52) << 23));
  bool ok = (E != 0) && (fe >= 1);
  bool okl = ok && (fe >= 53);
  df out;
  out.h = ok ? __uint_as_float(hbits) : 0.0f;
  out.l = okl ? __uint_as_float(__float_as_uint(l) ^ sign) : 0.0f;
  return out;
}

// Normalised df (h, l) -> binary64 bits: the magnitude of h as a 64-bit
// integer (Ed << 52 | significand) in units of ulp64(h), plus l expressed in
// the same units -- an exact power-of-two scaling, |l| < 2^28 units -- and
// rounded to an integer by F2I (round to nearest even).  When h is a power
// of two and l has the opposite sign the sum lies in the binade below, whose
// unit is half as large: there l is scaled by one more factor of two and the
// borrow from the exponent field lands the result in that binade.  Low parts
// of |h| < 2^-75 (relative to the scale) are dropped.
__device__ __forceinline__ void df_to_f64bits(df v, int D, uint32_t flip, uint32_t& olo, uint32_t& ohi) {
  v = df_norm(v);
  const uint32_t S = __float_as_uint(v.h), L = __float_as_uint(v.l);
  const uint32_t sign = (S ^ flip) & 0x80000000u;
  const int Es = (int)((S >> 23) & 0xFFu);
  const int Ed = Es + D;
  const bool down = ((S & 0x7FFFFFu) == 0u) && (((S ^ L) & 0x80000000u) != 0u);
  int lu = 0;
  if (Es >= 52)  // l * 2^(179-Es), or 2^(180-Es) in the binade below
    lu = __float2int_rn(__fmul_rn(v.l, __uint_as_float((uint32_t)(306 - Es + (down ? 1 : 0)) << 23)));
  if (S & 0x80000000u) lu = -lu;  // l relative to the sign of h
  const uint64_t mag =
      (((uint64_t)(uint32_t)Ed << 52) | ((uint64_t)(S & 0x7FFFFFu) << 29)) + (uint64_t)(int64_t)lu;
  uint32_t rh = (uint32_t)(mag >> 32), rl = (uint32_t)mag;
  const bool zero = (Es == 0) || (Ed <= 0);
  const bool inf = (Ed >= 2047) || ((rh >> 20) >= 2047u);
  if (zero) { rh = 0u; rl = 0u; }
  if (inf && !zero) { rh = 0x7FF00000u; rl = 0u; }
  ohi = sign | rh;
  olo = rl;
}

// ----------------------------------------------------------------------------
// Element loads / stores per policy and pass kind.
// ----------------------------------------------------------------------------
template <class P, int KIND>
struct Mem;

template <int KIND>
struct Mem<PolicyDF, KIND> {
  typedef uint4 Raw;
  static __device__ __forceinline__ cdf load(const void* base, uint64_t idx, int D, uint32_t conj) {
    if (KIND == FIRST || KIND == SINGLE) {
      // data is read once per pass: cache in L2 only (ld.global.cg) so that L1
      // keeps the twiddle tables; coherent at L2 (the buffer is written in place)
      uint4 v = __ldcg(reinterpret_cast<const uint4*>(base) + idx);
      cdf r;
      r.re = f64bits_to_df(v.x, v.y, D, 0u);
      r.im = f64bits_to_df(v.z, v.w, D, conj ? 0x80000000u : 0u);
      return r;
    } else {
      // intermediate double-float layout: {re.h, im.h, re.l, im.l}
      float4 v = __ldcg(reinterpret_cast<const float4*>(base) + idx);
      return cdf{{v.x, v.z}, {v.y, v.w}};
    }
  }
  static __device__ __forceinline__ void store(void* base, uint64_t idx, cdf x, int D, uint32_t conj,
                                               bool nonfinite) {
    if (KIND == LAST || KIND == SINGLE || KIND == LASTS) {
      uint4 o;
      df_to_f64bits(x.re, D, 0u, o.x, o.y);
      df_to_f64bits(x.im, D, conj ? 0x80000000u : 0u, o.z, o.w);
      if (nonfinite) o = make_uint4(0u, 0x7FF80000u, 0u, 0x7FF80000u);
      reinterpret_cast<uint4*>(base)[idx] = o;
    } else {
      df re = df_norm(x.re), im = df_norm(x.im);
      reinterpret_cast<float4*>(base)[idx] = make_float4(re.h, im.h, re.l, im.l);
    }
  }
};

template <int KIND>
struct Mem<PolicyDF2, KIND> {
  // an element's 16 bytes as stored in the buffer -> packed double-float
  static __device__ __forceinline__ cdf2 convert(uint4 v, int D, uint32_t conj) {
    if (KIND == FIRST || KIND == SINGLE) {
      df re = f64bits_to_df(v.x, v.y, D, 0u);
      df im = f64bits_to_df(v.z, v.w, D, conj ? 0x80000000u : 0u);
      return cdf2{make_float2(re.h, im.h), make_float2(re.l, im.l)};
    } else {
      return cdf2{make_float2(__uint_as_float(v.x), __uint_as_float(v.y)),
                  make_float2(__uint_as_float(v.z), __uint_as_float(v.w))};
    }
  }
  static __device__ __forceinline__ cdf2 load(const void* base, uint64_t idx, int D, uint32_t conj) {
    return convert(__ldcg(reinterpret_cast<const uint4*>(base) + idx), D, conj);
  }
  static __device__ __forceinline__ void store(void* base, uint64_t idx, cdf2 x, int D, uint32_t conj,
                                               bool nonfinite) {
    if (KIND == LAST || KIND == SINGLE || KIND == LASTS) {
      uint4 o;
      df_to_f64bits(df{x.h.x, x.l.x}, D, 0u, o.x, o.y);
      df_to_f64bits(df{x.h.y, x.l.y}, D, conj ? 0x80000000u : 0u, o.z, o.w);
      if (nonfinite) o = make_uint4(0u, 0x7FF80000u, 0u, 0x7FF80000u);
      reinterpret_cast<uint4*>(base)[idx] = o;
    } else {
      x = c2norm(x);
      reinterpret_cast<float4*>(base)[idx] = make_float4(x.h.x, x.h.y, x.l.x, x.l.y);
    }
  }
};

template <int KIND>
struct Mem<PolicyF32, KIND> {
  static __device__ __forceinline__ float2 load(const void* base, uint64_t idx, int, uint32_t conj) {
    float2 v = __ldcg(reinterpret_cast<const float2*>(base) + idx);
    if ((KIND == FIRST || KIND == SINGLE) && conj) v.y = -v.y;
    return v;
  }
  // D carries the output exponent shift for this policy: x * 2^-D
  static __device__ __forceinline__ void store(void* base, uint64_t idx, float2 x, int D, uint32_t conj, bool) {
    if (KIND == LAST || KIND == SINGLE || KIND == LASTS) {
      if (conj) x.y = -x.y;
      if (D) {
        const float sc = __uint_as_float((uint32_t)(127 - D) << 23);
        x.x = __fmul_rn(x.x, sc);
        x.y = __fmul_rn(x.y, sc);
      }
    }
    reinterpret_cast<float2*>(base)[idx] = x;
  }
};

__device__ __forceinline__ float4 ld_tw(const float4* t, uint32_t i) { return __ldg(t + i); }

// exp(-2*pi*i*idx/N) from the two-level table.
__device__ __forceinline__ float4 twiddle_N(const PassArgs& a, uint64_t idx) {
  uint32_t lo = (uint32_t)(idx & ((1ull << a.twB) - 1ull));
  uint32_t hi = (uint32_t)(idx >> a.twB);
  return tw_mul(ld_tw(a.tw_hi, hi), ld_tw(a.tw_lo, lo));
}

// Output digit k of position p inside a column (digit reversal over the
// pass's internal stages: nfull radix-16 stages, then radix 2^rem).
__device__ __forceinline__ int col_digit_reverse(int p, int log2R, int nfull, int rem) {
  int k = 0, shift = log2R;
#pragma unroll 1
  for (int st = 0; st < nfull; ++st) {
    shift -= 4;
    k |= ((p >> shift) & 15) << (4 * st);
  }
  if (rem) k |= (p & ((1 << rem) - 1)) << (4 * nfull);
  return k;
}

// Position (within the thread's 16 contiguous slots) of the output held in
// register u after the last stage: radix 16 (rem = 0) or 2^rem groups, each
// group's outputs in bit-reversed register order.
__device__ __forceinline__ int last_pos(int u, int rem) {
  if (rem == 0) return bitrev_n(u, 4);
  const int msk = (1 << rem) - 1;
  return (u & ~msk) | bitrev_n(u & msk, rem);
}

// ----------------------------------------------------------------------------
// The pass kernel.  C columns of R elements per CTA (C*R <= CTA_ELEMS), 16
// elements per thread, C*R/16 threads.  Thread tid = t*C + c handles column c.
// ----------------------------------------------------------------------------
template <class P, int KIND, int CTA_ELEMS>
__global__ void __launch_bounds__(CTA_ELEMS / 16, 2)
efft_pass(void* __restrict__ data, const PassArgs a) {
  typedef typename P::V V;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);

  const int log2R = a.log2R, log2C = a.log2C;
  const int R = 1 << log2R, C = 1 << log2C;
  const int tid = threadIdx.x;
  const int c = tid & (C - 1);
  const int t = tid >> log2C;  // 0 .. R/16 - 1
  const int nfull = log2R >> 2, rem = log2R & 3;
  const int nst = nfull + (rem ? 1 : 0);

  // column -> (block, m) -> element index of row 0
  const uint64_t jcol = (uint64_t)blockIdx.x * C + c;
  const uint64_t s = 1ull << a.log2s;
  const uint64_t m = jcol & (s - 1);
  const uint64_t colbase = ((jcol >> a.log2s) << a.log2L) + m;

  int D = 0, Dout = a.out_shift;
  bool nonfinite = false;
  if (P::kElemBytes == 16) {
    uint32_t emax = __ldg(state);
    D = (int)emax - 127;
    Dout = D - a.out_shift;
    nonfinite = (emax >= 0x7FFu);
  }

  V v[16];

  // ---- stage 0: straight from global memory ----
  {
    const int q = R >> 4;  // stride in rows
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = Mem<P, KIND>::load(data, colbase + ((uint64_t)(t + q * j) << a.log2s), D, a.conj_in);
  }

  // stages: radix-16 stages st = 0 .. nfull-1 (sub-block length l = R >> 4st),
  // then an optional radix-2^rem stage.  Stage st > 0 reads positions from
  // shared memory.
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    const bool last = (st == nst - 1);
    const bool small = last && rem;  // radix 2^rem stage on contiguous groups
    const int log2l = log2R - 4 * st;

    if (st > 0) {
      if (!small && !last) {
        const int log2g = log2l - 4;  // groups per sub-block = l/16
        const int b = t >> log2g, i = t & ((1 << log2g) - 1);
        const int p0 = (b << log2l) + i;
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = sm[smem_slot(p0 + (j << log2g), c, log2C)];
      } else {
        // last stage: the thread's 16 contiguous positions 16t .. 16t+15
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = sm[smem_slot((t << 4) + j, c, log2C)];
      }
    }

    if (!small) {
      dif_regs<P, 4>(v);
    } else if (rem == 1) {
#pragma unroll
      for (int u = 0; u < 8; ++u) dif_regs<P, 1>(v + 2 * u);
    } else if (rem == 2) {
#pragma unroll
      for (int u = 0; u < 4; ++u) dif_regs<P, 2>(v + 4 * u);
    } else {
#pragma unroll
      for (int u = 0; u < 2; ++u) dif_regs<P, 3>(v + 8 * u);
    }

    if (!last) {
      // internal twiddle exp(-2*pi*i * i*q / l), position i + (l/16) q in its
      // sub-block; register u holds q = bitrev4(u).
      const int log2g = log2l - 4;
      const int b = (st == 0) ? 0 : (t >> log2g);
      const int i = (st == 0) ? t : (t & ((1 << log2g) - 1));
      const int p0 = (b << log2l) + i;
      const int tshift = 11 - log2l;
#pragma unroll
      for (int u = 1; u < 16; ++u) {
        const int q = bitrev_n(u, 4);
        v[u] = P::mul_tw(v[u], ld_tw(a.w2048, (uint32_t)((i * q) << tshift)));
      }
      // in-place DIF: a thread writes exactly the 16 slots it read, so no
      // barrier is needed before the write, only before the next stage.
#pragma unroll
      for (int u = 0; u < 16; ++u) sm[smem_slot(p0 + (bitrev_n(u, 4) << log2g), c, log2C)] = v[u];
      __syncthreads();
    }
  }

  // ---- epilogue: digit-reversed positions -> output index k, pass twiddle,
  // store.  Register u holds position 16t + pos(u) of its column.
  if (a.log2s > 0) {
    // pass twiddle exp(-2*pi*i * m*k / L) = table index (m*k) << (log2N - log2L)
    const int sh = a.log2N - a.log2L;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = col_digit_reverse((t << 4) + last_pos(u, rem), log2R, nfull, rem);
      const uint64_t idx = ((uint64_t)m * (uint64_t)k) << sh;
      if (idx != 0) v[u] = P::mul_tw(v[u], twiddle_N(a, idx));
      Mem<P, KIND>::store(data, colbase + ((uint64_t)k << a.log2s), v[u], Dout, a.conj_out, nonfinite);
    }
  } else {
    // contiguous output: stage through shared memory in natural order
    if (nst > 1) __syncthreads();  // last-stage reads are complete
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = col_digit_reverse((t << 4) + last_pos(u, rem), log2R, nfull, rem);
      sm[smem_slot(k, c, log2C)] = v[u];
    }
    __syncthreads();
    const int tile_elems = R << log2C;  // C contiguous transforms
    const uint64_t tile0 = (uint64_t)blockIdx.x * tile_elems;
#pragma unroll 4
    for (int e = tid; e < tile_elems; e += (int)blockDim.x) {
      const int cc = e >> log2R, k = e & (R - 1);
      Mem<P, KIND>::store(data, tile0 + (uint64_t)e, sm[smem_slot(k, cc, log2C)], Dout, a.conj_out, nonfinite);
    }
  }
}

// ----------------------------------------------------------------------------
// Compile-time specialised pass kernel for the radices that carry the large
// sizes (R = 2^LR, LR = 8..11; C = 2^LC columns per CTA, C*R = CTA size).
// Same algorithm as efft_pass; with R and C known at compile time every
// shared-memory address is a per-thread base plus an immediate, and the pass
// twiddle exp(-2*pi*i*m*k/L) is factored as W_t * V_c[u]: k = kt | kc(u)
// (digit reversal is a bit permutation, so the thread's part kt and the
// register's part kc(u) occupy disjoint bits), W_t = exp(-2*pi*i*m*kt/L) is
// formed once per thread and V_c[u] = exp(-2*pi*i*m_c*kc(u)/L) once per column
// into shared memory, instead of two L2 table lookups per element.
// ----------------------------------------------------------------------------
__host__ __device__ constexpr int bitrev_c(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}
// output index k of column position p (see col_digit_reverse)
__host__ __device__ constexpr int digit_rev_c(int p, int LR) {
  int nfull = LR / 4, rem = LR % 4, k = 0, shift = LR;
  for (int st = 0; st < nfull; ++st) {
    shift -= 4;
    k |= ((p >> shift) & 15) << (4 * st);
  }
  if (rem) k |= (p & ((1 << rem) - 1)) << (4 * nfull);
  return k;
}
__host__ __device__ constexpr int last_pos_c(int u, int rem) {
  return rem == 0 ? bitrev_c(u, 4) : ((u & ~((1 << rem) - 1)) | bitrev_c(u & ((1 << rem) - 1), rem));
}
// padded slot offset of a raw offset that is a multiple of C (C a power of two)
__host__ __device__ constexpr int pad_off(int raw) { return raw + (raw >> 4); }

template <class P, int LOG>
__device__ __forceinline__ void dif_groups(typename P::V* v) {
  // 16 registers as 16 / 2^LOG independent radix-2^LOG DIF groups
#pragma unroll
  for (int g = 0; g < 16; g += (1 << LOG)) dif_regs<P, LOG>(v + g);
}

// Cluster-wide split barrier (all threads of both CTAs of a pair arrive,
// then wait): the hardware barrier of a thread-block cluster, whose CTAs are
// always resident together.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// The tile of a swapping middle pass (SWLT > 0).  The array is viewed as
// (i0, i1, i2) with i0 < A (stride L), i1 < R (stride A), i2 < A; a tile is
// the T x T block of columns i0 in [I T, I T + T), i2 in [J T, J T + T).  The
// CTA pair (cluster) z handles tiles (I, J) and (J, I), I < J, for
// z < nt (nt - 1) / 2 (nt = A / T), and the diagonal tiles (2d, 2d) and
// (2d + 1, 2d + 1), d = z - nt (nt - 1) / 2, after that.
__device__ __forceinline__ void swap_tile(uint32_t z, uint32_t rank, uint32_t nt, uint32_t& I, uint32_t& J) {
  const uint32_t P = nt * (nt - 1) / 2;
  if (z < P) {
    uint32_t j = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)z)) * 0.5f);
    while (j * (j - 1) / 2 > z) --j;
    while ((j + 1) * j / 2 <= z) ++j;
    const uint32_t i = z - j * (j - 1) / 2;
    I = rank ? j : i;
    J = rank ? i : j;
  } else {
    I = J = 2 * (z - P) + rank;
  }
}

// The specialised pass kernel (R = 2^LR rows, C = 2^LC columns per CTA,
// MINB CTAs per SM); grid.y selects the transform of a batched launch.
// SWLT > 0 (middle pass only, C = T^2 with T = 2^SWLT, launched as clusters
// of two CTAs): the pass also exchanges the outer digits, i.e. the result of
// column (i0, *, i2) is written to column (i2, *, i0), so that no separate
// digit-reversal sweep is needed.  The two CTAs of a cluster hold each
// other's destination tiles; a cluster barrier between their loads and their
// stores keeps the exchange in place.
template <class P, int KIND, int LR, int LC, int MINB = 2, int SWLT = 0>
__global__ void __launch_bounds__(1 << (LR + LC - 4), MINB)
efft_pass_fx(void* __restrict__ data, const PassArgs a) {
  typedef typename P::V V;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  constexpr int R = 1 << LR, C = 1 << LC, TPC = R >> 4, NT = (R * C) / 16;
  constexpr int NFULL = LR / 4, REM = LR % 4, NST = NFULL + (REM ? 1 : 0);
  constexpr int NMID = NST - 2;  // radix-16 stages between the first and the last
  constexpr bool SWAP = SWLT > 0;
  static_assert(!SWAP || (KIND == MID && LC == 2 * SWLT), "a swapping pass is a middle pass of T x T columns");
  constexpr bool STRIDED = (KIND == FIRST || KIND == MID || KIND == LASTS);
  constexpr bool TWID = (KIND == FIRST || KIND == MID);  // the pass twiddle of Eq. 4
  // Thread mapping: c runs fastest (a warp covers C columns x 32/C rows) and
  // shared memory is row-major, raw index p*C + c.  The last pass reads C
  // whole contiguous blocks: when a warp's run per column, 32/C elements,
  // would fill less than a 32-byte sector, t runs fastest instead (coalesced
  // loads) and shared memory is column-major, raw index c*R + p; its stage-0
  // twiddles then differ per lane, so it is used only there.  Either way
  // slot = raw + raw/16 (one pad slot per 16).
  constexpr bool CM = (KIND == LAST) && ((32 / C) * P::kElemBytes <= 32);
  constexpr int PS = CM ? 1 : C;  // raw step of one position p
  static_assert(LR >= 5 && LR <= 12, "radix range");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  __shared__ typename P::TW vtw[TWID ? 16 * C : 1];
  // column-major last pass: lanes hold different t, so the stage-0 twiddles
  // exp(-2*pi*i*t*q/R) come from a shared copy of the R-th roots of unity
  // (root k at k + k/8: lanes reading k = 8t or 4t stay on different banks)
  __shared__ float4 wroot[CM ? R + R / 8 : 1];
  auto slot = [](int p, int col) {
    const int raw = CM ? (col << LR) + p : (p << LC) + col;
    return raw + (raw >> 4);
  };

  const int tid = threadIdx.x;
  const int c = CM ? (tid >> (LR - 4)) : (tid & (C - 1));
  const int t = CM ? (tid & (TPC - 1)) : (tid >> LC);
  const uint64_t jcol = (uint64_t)blockIdx.x * C + c;
  uint64_t m = 0, colbase, step, outbase = 0;
  uint32_t tI = 0, tJ = 0;  // swapping pass: this CTA's tile
  if (SWAP) {
    constexpr int T = 1 << SWLT;
    swap_tile(blockIdx.x >> 1, blockIdx.x & 1, 1u << (a.log2s - SWLT), tI, tJ);
    const uint64_t i0 = (uint64_t)tI * T + (c >> SWLT), i2 = (uint64_t)tJ * T + (c & (T - 1));
    step = 1ull << a.log2s;
    m = i2;
    colbase = (i0 << a.log2L) + i2;
    outbase = (i2 << a.log2L) + i0;
  } else if (KIND == FIRST || KIND == LASTS) {
    // the first pass spans the whole array (L = N): column j starts at j;
    // so does the strided last pass (the columns of the swapped layout)
    step = (KIND == FIRST ? (uint64_t)a.s_odd : 1ull) << a.log2s;
    m = jcol;
    colbase = jcol;
  } else if (STRIDED) {
    step = 1ull << a.log2s;
    m = jcol & (step - 1);
    colbase = ((jcol >> a.log2s) << a.log2L) + m;
  } else {
    step = 1;
    colbase = jcol << LR;
  }

  int D = 0, Dout = a.out_shift;
  bool nonfinite = false;
  if (P::kElemBytes == 16) {
    uint32_t emax = __ldg(state);
    D = (int)emax - 127;
    Dout = D - a.out_shift;
    nonfinite = (emax >= 0x7FFu);
  }

  const int kt = digit_rev_c(t << 4, LR);
  typename P::TW wt;
  if (TWID) {
    const int sh = (KIND == FIRST) ? 0 : a.log2N - a.log2L;
    // V_c[u] stored as [u][c]: the columns of one warp read consecutive entries
    if (tid < 16 * C) {
      const int cc = tid >> 4, u = tid & 15;
      const uint64_t mc = SWAP ? (uint64_t)tJ * (1u << SWLT) + (cc & ((1 << SWLT) - 1))
                               : ((uint64_t)blockIdx.x * C + cc) & (KIND == FIRST ? ~0ull : step - 1);
      const int kc = digit_rev_c(last_pos_c(u, REM), LR);
      vtw[u * C + cc] = P::expand(twiddle_N(a, (mc * (uint64_t)kc) << sh));
    }
    wt = P::expand(twiddle_N(a, (m * (uint64_t)kt) << sh));
  }

  V v[16];
  // ---- stage 0: rows t + TPC*j straight from global memory ----
  {
    const uint64_t b0 = colbase + (uint64_t)t * step, sj = (uint64_t)TPC * step;
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = Mem<P, KIND>::load(data, b0 + (uint64_t)j * sj, D, a.conj_in);
  }
  if (CM) {
    for (int k = tid; k < R; k += NT) wroot[k + (k >> 3)] = __ldg(a.w2048 + (k << (11 - LR)));
    __syncthreads();
  }
  dif_regs<P, 4>(v);
  // the stage-0 loads are consumed: the partner CTA may overwrite this tile
  if (SWAP) cluster_arrive();
  {
    // exp(-2*pi*i * t*q / R), q = bitrev4(u), to positions t + TPC*q
#pragma unroll
    for (int u = 1; u < 16; ++u)
      v[u] = P::mul_tw(v[u], CM ? P::expand(wroot[t * bitrev_c(u, 4) + ((t * bitrev_c(u, 4)) >> 3)])
                                : P::int_tw(a.w2048, nullptr, (uint32_t)(t * bitrev_c(u, 4)) << (11 - LR)));
    const int sb = slot(t, c);
#pragma unroll
    for (int u = 0; u < 16; ++u) sm[sb + pad_off(bitrev_c(u, 4) * TPC * PS)] = v[u];
  }
  __syncthreads();

  // ---- middle radix-16 stages ----
#pragma unroll
  for (int st = 1; st <= NMID; ++st) {
    const int log2l = LR - 4 * st;      // sub-block length
    const int log2g = log2l - 4;        // groups per sub-block
    const int b = t >> log2g, i = t & ((1 << log2g) - 1);
    const int sb = slot((b << log2l) + i, c);
    const int gstep = (1 << log2g) * PS;  // raw step between group members
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = sm[sb + pad_off(j * gstep)];
    dif_regs<P, 4>(v);
#pragma unroll
    for (int u = 1; u < 16; ++u)
      v[u] = P::mul_tw(v[u], P::int_tw(a.w2048, nullptr, (uint32_t)(i * bitrev_c(u, 4)) << (11 - log2l)));
    // in place: the thread writes exactly the slots it read
#pragma unroll
    for (int u = 0; u < 16; ++u) sm[sb + pad_off(bitrev_c(u, 4) * gstep)] = v[u];
    __syncthreads();
  }

  // ---- last stage: the thread's 16 contiguous positions 16t .. 16t+15 ----
  {
    const int sb = slot(t << 4, c);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = sm[sb + pad_off(j * PS)];
    if (REM == 0) dif_regs<P, 4>(v);
    else dif_groups<P, (REM == 0 ? 4 : REM)>(v);
  }

  if (STRIDED && (KIND != FIRST || a.s_odd == 1)) {
    // swapping pass: the partner CTA has consumed its loads of this CTA's
    // destination tile
    if (SWAP) cluster_wait();
    const uint64_t ob = SWAP ? outbase : colbase;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = kt | digit_rev_c(last_pos_c(u, REM), LR);
      if (TWID) v[u] = P::pass_tw(v[u], wt, vtw[u * C + c]);
      Mem<P, KIND>::store(data, ob + ((uint64_t)k << a.log2s), v[u], Dout, a.conj_out, nonfinite);
    }
  } else if (STRIDED) {
    // first pass of N = M * 2^e: output k at k * M * 2^log2s
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = kt | digit_rev_c(last_pos_c(u, REM), LR);
      v[u] = P::pass_tw(v[u], wt, vtw[u * C + c]);
      Mem<P, KIND>::store(data, colbase + ((uint64_t)(k * a.s_odd) << a.log2s), v[u], Dout, a.conj_out,
                          nonfinite);
    }
  } else {
    __syncthreads();  // last-stage reads are complete before the slots are reused
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = kt | digit_rev_c(last_pos_c(u, REM), LR);
      sm[slot(k, c)] = v[u];
    }
    __syncthreads();
    const uint64_t tile0 = (uint64_t)blockIdx.x * (R * C);
#pragma unroll 4
    for (int e = tid; e < R * C; e += NT) {
      const int cc = e >> LR, k = e & (R - 1);
      Mem<P, KIND>::store(data, tile0 + (uint64_t)e, sm[slot(k, cc)], Dout, a.conj_out, nonfinite);
    }
  }
}

// ----------------------------------------------------------------------------
// Persistent complex128 strided pass with the next tile's loads in flight
// during the current tile's last stage and epilogue.
//
// A strided pass kernel of one CTA per tile loads its tile, then computes;
// with one or two CTAs per SM (the register file holds only that many
// 16-value double-float threads) the FP32 pipe idles while a new CTA's loads
// are outstanding.  Here each CTA walks tiles tile, tile + grid, ...; as soon
// as every thread has read the last stage's inputs from shared memory the
// buffer is free, and each thread issues asynchronous copies (cp.async, 16
// bytes each, cached in L2 only) of its own 16 stage-0 elements of the next
// tile into their shared-memory slots.  Those copies complete while the last
// stage, the pass twiddle and the stores run; the next tile then starts from
// shared memory.  Same arithmetic, same results as efft_pass_fx.
// Kinds: FIRST (power-of-two N), MID (also swapping, SWLT > 0), LASTS.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const size_t ga = __cvta_generic_to_global(gmem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(ga) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Column geometry of a strided pass: first element, row step, twiddle index
// m and output base of column c of tile `tile` (a swapping pass: of the
// rank-th tile of tile pair `tile`).
struct Geo {
  uint64_t colbase, step, m, outbase;
};
template <int KIND, int LC, int SWLT>
__device__ __forceinline__ Geo strided_geo(const PassArgs& a, uint64_t tile, uint32_t rank, int c) {
  Geo g;
  g.step = 1ull << a.log2s;
  if (SWLT > 0) {
    constexpr int T = 1 << SWLT;
    uint32_t I, J;
    swap_tile((uint32_t)tile, rank, 1u << (a.log2s - SWLT), I, J);
    const uint64_t i0 = (uint64_t)I * T + (c >> SWLT), i2 = (uint64_t)J * T + (c & (T - 1));
    g.m = i2;
    g.colbase = (i0 << a.log2L) + i2;
    g.outbase = (i2 << a.log2L) + i0;
  } else if (KIND == FIRST || KIND == LASTS) {
    const uint64_t jcol = (tile << LC) + c;
    g.m = jcol;
    g.colbase = g.outbase = jcol;
  } else {
    const uint64_t jcol = (tile << LC) + c;
    g.m = jcol & (g.step - 1);
    g.colbase = g.outbase = ((jcol >> a.log2s) << a.log2L) + g.m;
  }
  return g;
}

template <int KIND, int LR, int LC, int MINB, int SWLT = 0>
__global__ void __launch_bounds__(1 << (LR + LC - 4), MINB)
efft_pass_pf(void* __restrict__ data, const PassArgs a) {
  typedef PolicyDF2 P;
  typedef P::V V;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  constexpr int R = 1 << LR, C = 1 << LC, TPC = R >> 4;
  constexpr int NFULL = LR / 4, REM = LR % 4, NST = NFULL + (REM ? 1 : 0);
  constexpr int NMID = NST - 2;
  constexpr bool SWAP = SWLT > 0;
  constexpr bool TWID = (KIND == FIRST || KIND == MID);
  static_assert(KIND == FIRST || KIND == MID || KIND == LASTS, "strided kinds only");
  static_assert(!SWAP || (KIND == MID && LC == 2 * SWLT), "a swapping pass is a middle pass of T x T columns");
  static_assert(LR >= 5 && LR <= 12, "radix range");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  __shared__ P::TW vtw[TWID ? 16 * C : 1];
  auto slot = [](int p, int col) {
    const int raw = (p << LC) + col;
    return raw + (raw >> 4);
  };

  const int tid = threadIdx.x;
  const int c = tid & (C - 1);
  const int t = tid >> LC;
  const uint32_t emax = __ldg(state);
  const int D = (int)emax - 127;
  const int Dout = D - a.out_shift;
  const bool nonfinite = (emax >= 0x7FFu);
  const int kt = digit_rev_c(t << 4, LR);
  const int sb0 = slot(t, c);  // the thread's stage-0 slots: sb0 + pad_off(j * TPC * C)

  const uint32_t rank = SWAP ? (blockIdx.x & 1u) : 0u;
  const uint64_t stride = SWAP ? (gridDim.x >> 1) : gridDim.x;
  uint64_t tile = SWAP ? (blockIdx.x >> 1) : blockIdx.x;

  // the thread's 16 stage-0 elements of `tl`, rows t + TPC*j, into their slots
  auto prefetch = [&](uint64_t tl) {
    const Geo g = strided_geo<KIND, LC, SWLT>(a, tl, rank, c);
    const uint64_t b0 = g.colbase + (uint64_t)t * g.step, sj = (uint64_t)TPC * g.step;
    const uint4* src = reinterpret_cast<const uint4*>(data);
#pragma unroll
    for (int j = 0; j < 16; ++j) cp_async16(&sm[sb0 + pad_off(j * TPC * C)], src + b0 + (uint64_t)j * sj);
    cp_async_commit();
  };
  if (tile < a.ntiles) prefetch(tile);

  for (; tile < a.ntiles; tile += stride) {
    const Geo g = strided_geo<KIND, LC, SWLT>(a, tile, rank, c);
    __syncthreads();  // the previous tile's epilogue no longer reads vtw
    P::TW wt;
    if (TWID) {
      const int sh = (KIND == FIRST) ? 0 : a.log2N - a.log2L;
      if (tid < 16 * C) {
        const int cc = tid >> 4, u = tid & 15;
        const uint64_t mc = strided_geo<KIND, LC, SWLT>(a, tile, rank, cc).m;
        const int kc = digit_rev_c(last_pos_c(u, REM), LR);
        vtw[u * C + cc] = P::expand(twiddle_N(a, (mc * (uint64_t)kc) << sh));
      }
      wt = P::expand(twiddle_N(a, (g.m * (uint64_t)kt) << sh));
    }

    V v[16];
    // ---- stage 0: the thread's own copies, now in shared memory ----
    cp_async_wait_all();
#pragma unroll
    for (int j = 0; j < 16; ++j)
      v[j] = Mem<P, KIND>::convert(reinterpret_cast<const uint4*>(sm)[sb0 + pad_off(j * TPC * C)], D, a.conj_in);
    dif_regs<P, 4>(v);
    // this tile's global loads are complete: the partner CTA may overwrite it
    if (SWAP) cluster_arrive();
#pragma unroll
    for (int u = 1; u < 16; ++u)
      v[u] = P::mul_tw(v[u], P::int_tw(a.w2048, nullptr, (uint32_t)(t * bitrev_c(u, 4)) << (11 - LR)));
#pragma unroll
    for (int u = 0; u < 16; ++u) sm[sb0 + pad_off(bitrev_c(u, 4) * TPC * C)] = v[u];
    __syncthreads();

    // ---- middle radix-16 stages ----
#pragma unroll
    for (int st = 1; st <= NMID; ++st) {
      const int log2l = LR - 4 * st;
      const int log2g = log2l - 4;
      const int b = t >> log2g, i = t & ((1 << log2g) - 1);
      const int sb = slot((b << log2l) + i, c);
      const int gstep = (1 << log2g) * C;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = sm[sb + pad_off(j * gstep)];
      dif_regs<P, 4>(v);
#pragma unroll
      for (int u = 1; u < 16; ++u)
        v[u] = P::mul_tw(v[u], P::int_tw(a.w2048, nullptr, (uint32_t)(i * bitrev_c(u, 4)) << (11 - log2l)));
#pragma unroll
      for (int u = 0; u < 16; ++u) sm[sb + pad_off(bitrev_c(u, 4) * gstep)] = v[u];
      __syncthreads();
    }

    // ---- last stage; then the buffer is free for the next tile's copies ----
    {
      const int sb = slot(t << 4, c);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = sm[sb + pad_off(j * C)];
    }
    __syncthreads();
    if (tile + stride < a.ntiles) prefetch(tile + stride);
    if (REM == 0) dif_regs<P, 4>(v);
    else dif_groups<P, (REM == 0 ? 4 : REM)>(v);

    if (SWAP) cluster_wait();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = kt | digit_rev_c(last_pos_c(u, REM), LR);
      if (TWID) v[u] = P::pass_tw(v[u], wt, vtw[u * C + c]);
      Mem<P, KIND>::store(data, g.outbase + ((uint64_t)k << a.log2s), v[u], Dout, a.conj_out, nonfinite);
    }
  }
  cp_async_wait_all();  // nothing is left in flight when the CTA exits
}

// ----------------------------------------------------------------------------
// N <= 8: one thread, Eq. 1 evaluated directly with table twiddles.
// ----------------------------------------------------------------------------
template <class P>
__global__ void efft_small(void* __restrict__ data, const PassArgs a) {
  typedef typename P::V V;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  const int N = 1 << a.log2N;
  int D = 0, Dout = a.out_shift;
  bool nonfinite = false;
  if (P::kElemBytes == 16) {
    uint32_t emax = __ldg(state);
    D = (int)emax - 127;
    Dout = D - a.out_shift;
    nonfinite = (emax >= 0x7FFu);
  }
  V x[8], y[8];
  for (int n = 0; n < N; ++n) x[n] = Mem<P, SINGLE>::load(data, n, D, a.conj_in);
  for (int k = 0; k < N; ++k) {
    V acc = x[0];
    for (int n = 1; n < N; ++n) {
      int t = ((n * k) & (N - 1)) << (11 - a.log2N);
      acc = P::add(acc, P::mul_tw(x[n], ld_tw(a.w2048, t)));
    }
    y[k] = acc;
  }
  for (int k = 0; k < N; ++k) Mem<P, SINGLE>::store(data, k, y[k], Dout, a.conj_out, nonfinite);
}

// Launch interface of the specialised kernels (one translation unit per
// policy, compiled in parallel): efft_fx_df2.cu (complex128, packed
// double-float), efft_fx_f32.cu (complex64).
cudaError_t fx_set_attrs_df2();
bool fx_launch_df2(int kind, int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                   const PassArgs& a);
// complex128 first pass with 8192-element tiles (R = 2^10 or 2^11), one CTA
// of 512 threads per SM: twice the bytes per row segment of the 4096-element
// tile, for first passes whose rows lie in different pages.
constexpr int kLog2CtaWide = 13;
bool fx_launch_df2_wide(int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                        const PassArgs& a);
// complex128 passes of a three-pass schedule whose middle pass swaps the
// outer digits (clusters of two CTAs) and whose last pass is strided:
// the middle pass of R = 2^log2R rows on T x T column tiles and the last
// pass of R = 2^9..2^11 rows on 8192-element tiles (one CTA per SM).
bool fx_launch_df2_swap(int log2R, int log2C, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                        const PassArgs& a);
bool fx_launch_df2_lasts(int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                         const PassArgs& a);
// complex128 strided passes as persistent kernels (efft_pass_pf): `grid`
// CTAs walk a.ntiles tiles (tile pairs for a swapping pass, swap > 0).
cudaError_t fx_set_attrs_df2_pf();
bool fx_launch_df2_pf(int kind, int log2R, int log2C, int swap, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      void* data, const PassArgs& a);
cudaError_t fx_set_attrs_f32();
bool fx_launch_f32(int kind, int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                   const PassArgs& a);
// complex64 passes on 16384-element tiles, one CTA per SM: the first pass of
// R = 2^10 rows (radix-32 kernel, 16 columns, 128 bytes per row segment) and
// the middle pass of R = 2^11 rows (8 columns, 64 bytes per row segment).
constexpr int kLog2CtaWideC64 = 14;
bool fx_launch_f32_wide(int kind, int log2R, dim3 grid, cudaStream_t st, void* data, const PassArgs& a);
// the wide complex64 first pass (R = 2^10, 16 columns) as a persistent kernel
// fed by TMA copies; tensor_map: a CUtensorMap of the array as [1024][N/1024]
// 8-byte elements with 16 x 256 boxes.  `grid` CTAs walk a.ntiles tiles.
bool fx_launch_f32_tma(dim3 grid, cudaStream_t st, void* data, const PassArgs& a, const void* tensor_map);

}  // namespace efft
