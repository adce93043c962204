// efft_mix.cuh -- the mixed-radix pass kernel for N = M * 2^e (M odd).
// Included by efft_mix.cu only.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "efft_kernels.cuh"

namespace efft {

// ----------------------------------------------------------------------------
// Mixed-radix pass for N = M * 2^e (M odd, the paper's size set of Sec. 2.1):
// the same in-place pass as efft_pass (a batch of strided size-R DFTs and
// the twiddle of Eq. 4), for any radix R = M' * 2^b (M' = 1 or M) and any
// integer stride and block length.  The R-point DFT of each column is a
// mixed-radix Stockham (self-sorting) sequence in shared memory: radices
// 16, 8, 4, 2 and the odd factor, ping-ponging between two buffers, so every
// column ends in natural order; odd radices are direct sums.  The R-th roots
// of unity are computed once per CTA into shared memory and serve every
// stage twiddle and the odd radix; the pass twiddle exp(-2*pi*i*m*q/L) comes
// from the two-level table of exp(-2*pi*i*idx/N) (idx = m*q*N/L < N).
// ----------------------------------------------------------------------------
struct MixArgs {
  uint64_t N;      // transform length
  uint64_t s, L;   // column stride and block length of this pass
  int R, C;        // radix and columns per CTA (C a power of two dividing s)
  int log2C;
  int nrad;        // Stockham stages
  int rad[8];      // their radices (product R)
  int twB;         // low-table bits of the two-level table
  const float4* tw_lo;
  const float4* tw_hi;
  const uint32_t* state;
  void* const* ptrs;
  uint32_t conj_in, conj_out;
  int out_shift;
  int log2b, log2s;  // middle-pass kernel: R = M * 2^log2b, s = 2^log2s
};

__device__ __forceinline__ float4 twiddle_mix(const MixArgs& a, uint64_t idx) {
  return tw_mul(__ldg(a.tw_hi + (idx >> a.twB)), __ldg(a.tw_lo + (idx & ((1ull << a.twB) - 1ull))));
}

// Shared-memory slot of buffer index i: one pad slot per 16, so the
// stride-p writes of a stage (p = 16 at Ns = 1) spread over the banks.
__device__ __forceinline__ int mix_slot(int i) { return i + (i >> 4); }

// One Stockham stage of radix p over the C columns of a tile: work item
// (column c, j < R/p) reads v[r] = in[j + r R/p], multiplies by
// exp(-2*pi*i*k*r/(Ns p)) = roots[k r R/(Ns p)] (k = j mod Ns), takes the
// p-point DFT Y[q] = sum_r v[r] exp(-2*pi*i*q*r/p) (roots[q r R/p]) and
// writes Y[q] to out[(j/Ns) Ns p + k + q Ns].  Radices 8 and 16 run the
// in-register DIF butterflies of the power-of-two passes, 2 and 4 direct
// butterflies; an odd radix is a direct sum whose outputs go straight to
// shared memory one by one (only the p inputs stay in registers).
template <class P, int p>
__device__ __forceinline__ void mix_stage(const typename P::V* in, typename P::V* out, int R, int C, int Ns,
                                          const float4* roots) {
  typedef typename P::V V;
  const int Rp = R / p, tstep = R / (Ns * p);
  for (int w = threadIdx.x; w < C * Rp; w += blockDim.x) {
    const int c = w / Rp, j = w - c * Rp, k = j % Ns;
    V v[p];
#pragma unroll
    for (int r = 0; r < p; ++r) v[r] = in[mix_slot(c * R + j + r * Rp)];
    if (k) {
#pragma unroll
      for (int r = 1; r < p; ++r) v[r] = P::mul_tw(v[r], P::expand(roots[k * r * tstep]));
    }
    const int ob = c * R + (j / Ns) * Ns * p + k;  // output q at ob + q*Ns
    if (p == 8 || p == 16) {
      // in-register decimation in frequency: register u holds Y[bitrev(u)]
      constexpr int LOG = (p == 16) ? 4 : 3;
      dif_regs<P, LOG>(v);
#pragma unroll
      for (int u = 0; u < p; ++u) out[mix_slot(ob + bitrev_c(u, LOG) * Ns)] = v[u];
    } else if (p == 2) {
      out[mix_slot(ob)] = P::add(v[0], v[1]);
      out[mix_slot(ob + Ns)] = P::sub(v[0], v[1]);
    } else if (p == 4) {
      const V s02 = P::add(v[0], v[2]), d02 = P::sub(v[0], v[2]);
      const V s13 = P::add(v[1], v[3]), d13 = P::mul_negi(P::sub(v[1], v[3]));
      out[mix_slot(ob)] = P::add(s02, s13);
      out[mix_slot(ob + 2 * Ns)] = P::sub(s02, s13);
      out[mix_slot(ob + Ns)] = P::add(d02, d13);
      out[mix_slot(ob + 3 * Ns)] = P::sub(d02, d13);
    } else {
      V acc = v[0];
#pragma unroll
      for (int r = 1; r < p; ++r) acc = P::add(acc, v[r]);
      out[mix_slot(ob)] = acc;
#pragma unroll 1
      for (int q = 1; q < p; ++q) {
        acc = v[0];
#pragma unroll
        for (int r = 1; r < p; ++r) acc = P::add(acc, P::mul_tw(v[r], P::expand(roots[((q * r) % p) * Rp])));
        out[mix_slot(ob + q * Ns)] = acc;
      }
    }
  }
}

// Threads per CTA and elements per thread of the tile load and store
// (tiles of at most 2048 elements).
constexpr int kMixThreads = 256;
constexpr int kMixPerThread = 8;

// Dynamic shared memory: two padded buffers of C*R values, then R roots.
template <class P, int KIND>
__global__ void __launch_bounds__(kMixThreads, 2) efft_pass_mix(void* __restrict__ data, const MixArgs a) {
  typedef typename P::V V;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = a.R, C = a.C, CR = R * C, CRP = CR + CR / 16;
  V* in = reinterpret_cast<V*>(smem_raw);
  V* out = in + CRP;
  float4* roots = reinterpret_cast<float4*>(out + CRP);

  int D = 0, Dout = a.out_shift;
  bool nonfinite = false;
  if (P::kElemBytes == 16) {
    const uint32_t emax = __ldg(state);
    D = (int)emax - 127;
    Dout = D - a.out_shift;
    nonfinite = (emax >= 0x7FFu);
  }
  // exp(-2*pi*i*j/R), j < R
  const uint64_t runit = a.N / (uint64_t)R;
  for (int j = threadIdx.x; j < R; j += blockDim.x) roots[j] = twiddle_mix(a, (uint64_t)j * runit);

  // The CTA's columns jcol0 .. jcol0 + C - 1 lie in one block (C divides s):
  // column jcol0 + c, row r is at base0 + c * cstep + r * s.
  const uint64_t jcol0 = (uint64_t)blockIdx.x * C;
  const uint64_t blk = jcol0 / a.s, m0 = jcol0 - blk * a.s;
  const uint64_t base0 = blk * a.L + m0;
  const bool strided = (a.s > 1);
  const uint64_t cstep = strided ? 1ull : a.L;
  // load: adjacent threads read adjacent columns of a row (strided) or
  // adjacent elements of a column (contiguous blocks); all of a thread's
  // loads are issued before the first shared-memory write
  auto rc_of = [&](int e, int& r, int& c) {
    if (strided) {
      r = e >> a.log2C;
      c = e & (C - 1);
    } else {
      c = e / R;
      r = e - c * R;
    }
  };
  {
    V x[kMixPerThread];
#pragma unroll
    for (int i = 0; i < kMixPerThread; ++i) {
      const int e = threadIdx.x + i * kMixThreads;
      int r = 0, c = 0;
      rc_of(e, r, c);
      if (e < CR) x[i] = Mem<P, KIND>::load(data, base0 + c * cstep + (uint64_t)r * a.s, D, a.conj_in);
    }
#pragma unroll
    for (int i = 0; i < kMixPerThread; ++i) {
      const int e = threadIdx.x + i * kMixThreads;
      int r = 0, c = 0;
      rc_of(e, r, c);
      if (e < CR) in[mix_slot(c * R + r)] = x[i];
    }
  }
  __syncthreads();

  int Ns = 1;
  for (int st = 0; st < a.nrad; ++st) {
    const int p = a.rad[st];
    switch (p) {
      case 2: mix_stage<P, 2>(in, out, R, C, Ns, roots); break;
      case 4: mix_stage<P, 4>(in, out, R, C, Ns, roots); break;
      case 8: mix_stage<P, 8>(in, out, R, C, Ns, roots); break;
      case 16: mix_stage<P, 16>(in, out, R, C, Ns, roots); break;
      case 3: mix_stage<P, 3>(in, out, R, C, Ns, roots); break;
      case 5: mix_stage<P, 5>(in, out, R, C, Ns, roots); break;
      case 7: mix_stage<P, 7>(in, out, R, C, Ns, roots); break;
      case 9: mix_stage<P, 9>(in, out, R, C, Ns, roots); break;
      case 11: mix_stage<P, 11>(in, out, R, C, Ns, roots); break;
      case 13: mix_stage<P, 13>(in, out, R, C, Ns, roots); break;
      default: mix_stage<P, 15>(in, out, R, C, Ns, roots); break;
    }
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
    Ns *= p;
  }

  // epilogue: in[c*R + q] holds X[q] of column c; the pass twiddle
  // exp(-2*pi*i*m*q/L) on strided passes, then the store
  const uint64_t tw_unit = a.N / a.L;
  {
    // twiddle lookups of all the thread's elements first, then the stores
    float4 w[kMixPerThread];
#pragma unroll
    for (int i = 0; i < kMixPerThread; ++i) {
      const int e = threadIdx.x + i * kMixThreads;
      int r = 0, c = 0;
      rc_of(e, r, c);
      const uint64_t m = strided ? m0 + c : 0;
      if (e < CR && m != 0 && r != 0) w[i] = twiddle_mix(a, m * (uint64_t)r * tw_unit);
    }
#pragma unroll
    for (int i = 0; i < kMixPerThread; ++i) {
      const int e = threadIdx.x + i * kMixThreads;
      int r = 0, c = 0;
      rc_of(e, r, c);
      if (e < CR) {
        V v = in[mix_slot(c * R + r)];
        const uint64_t m = strided ? m0 + c : 0;
        if (m != 0 && r != 0) v = P::mul_tw(v, P::expand(w[i]));
        Mem<P, KIND>::store(data, base0 + c * cstep + (uint64_t)r * a.s, v, Dout, a.conj_out, nonfinite);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Middle pass of N = M * 2^e with the odd factor M fixed at compile time:
// R = M * 2^b (b >= 4), stride s = 2^log2s, C = 2^log2C <= 32 columns per
// CTA.  The same Stockham sequence as efft_pass_mix with the power-of-two
// stages first (radix 8, then one of 2 or 4: Ns is a power of two and the
// index arithmetic shifts; radix-16 stages spill at two CTAs per SM and
// measured slower) and the odd stages last (9 = 3*3, 15 = 3*5); radix 3 is
// the butterfly
//   Y0 = v0 + t1, Y1,2 = v0 - t1/2 -/+ i (sqrt(3)/2)(v1 - v2), t1 = v1 + v2,
// the others direct sums.  The pass twiddle exp(-2*pi*i*m*r/L) is factored
// as in efft_pass_fx: a thread's elements r = r0 + i*RS of column c
// (RS = threads / C) take W(m r0) * W(m RS i), the first formed once per
// thread, the second from a table of kMixPerThread entries per column.
// ----------------------------------------------------------------------------
template <int M> struct MixOdd { static constexpr int p0 = M, p1 = 1; };
template <> struct MixOdd<9> { static constexpr int p0 = 3, p1 = 3; };
template <> struct MixOdd<15> { static constexpr int p0 = 3, p1 = 5; };

// x times the real double-float constant c
__device__ __forceinline__ cdf2 mix_scale(cdf2 x, df c) { return c2mulr(x, c); }
__device__ __forceinline__ float2 mix_scale(float2 x, df c) {
  return make_float2(__fmaf_rn(x.x, c.h, __fmul_rn(x.x, c.l)), __fmaf_rn(x.y, c.h, __fmul_rn(x.y, c.l)));
}
__device__ __forceinline__ df K_SQRT3_2() { return {0x1.bb67aep-1f, 0x1.0b0996p-26f}; }  // sqrt(3)/2

// Power-of-two Stockham stage of radix Q = 2^LQ at Ns = 2^ls (see mix_stage).
template <class P, int M, int LQ>
__device__ __forceinline__ void mixm_pow2_stage(const typename P::V* in, typename P::V* out, int b, int lc, int ls,
                                                const float4* roots) {
  typedef typename P::V V;
  constexpr int Q = 1 << LQ;
  const int lrq = b - LQ, RQ = M << lrq, R = M << b;  // R/Q = M * 2^lrq
  const int tsh = b - ls - LQ;                        // R/(Ns Q) = M * 2^tsh
  const int items = RQ << lc, Ns = 1 << ls;
  for (int w = threadIdx.x; w < items; w += kMixThreads) {
    const int c = (w >> lrq) / M;
    const int j = w - c * RQ;
    const int k = j & (Ns - 1);
    V v[Q];
#pragma unroll
    for (int r = 0; r < Q; ++r) v[r] = in[mix_slot(c * R + j + r * RQ)];
    if (k) {
#pragma unroll
      for (int r = 1; r < Q; ++r) v[r] = P::mul_tw(v[r], P::expand(roots[(k * r * M) << tsh]));
    }
    const int ob = c * R + ((j - k) << LQ) + k;  // (j/Ns) Ns Q + k
    if constexpr (Q >= 8) {
      dif_regs<P, LQ>(v);
#pragma unroll
      for (int u = 0; u < Q; ++u) out[mix_slot(ob + bitrev_c(u, LQ) * Ns)] = v[u];
    } else if constexpr (Q == 4) {
      const V s02 = P::add(v[0], v[2]), d02 = P::sub(v[0], v[2]);
      const V s13 = P::add(v[1], v[3]), d13 = P::mul_negi(P::sub(v[1], v[3]));
      out[mix_slot(ob)] = P::add(s02, s13);
      out[mix_slot(ob + 2 * Ns)] = P::sub(s02, s13);
      out[mix_slot(ob + Ns)] = P::add(d02, d13);
      out[mix_slot(ob + 3 * Ns)] = P::sub(d02, d13);
    } else {
      out[mix_slot(ob)] = P::add(v[0], v[1]);
      out[mix_slot(ob + Ns)] = P::sub(v[0], v[1]);
    }
  }
}

// Odd Stockham stage of radix PO after odd stages of product PREV:
// Ns = PREV * 2^b, R/PO = (M/PO) * 2^b.
template <class P, int M, int PO, int PREV>
__device__ __forceinline__ void mixm_odd_stage(const typename P::V* in, typename P::V* out, int b, int lc,
                                               const float4* roots) {
  typedef typename P::V V;
  constexpr int RQM = M / PO, TST = M / (PREV * PO);  // R/(Ns PO) = TST
  const int R = M << b, RQ = RQM << b, Ns = PREV << b;
  const int items = RQ << lc;
  for (int w = threadIdx.x; w < items; w += kMixThreads) {
    const int c = (w >> b) / RQM;
    const int j = w - c * RQ;
    const int jq = (j >> b) / PREV;  // j / Ns
    const int k = j - jq * Ns;
    V v[PO];
#pragma unroll
    for (int r = 0; r < PO; ++r) v[r] = in[mix_slot(c * R + j + r * RQ)];
    if (k) {
#pragma unroll
      for (int r = 1; r < PO; ++r) v[r] = P::mul_tw(v[r], P::expand(roots[k * r * TST]));
    }
    const int ob = c * R + jq * Ns * PO + k;
    if constexpr (PO == 3) {
      const V t1 = P::add(v[1], v[2]);
      const V t2 = P::sub(v[0], mix_scale(t1, df{0.5f, 0.f}));
      const V t3 = P::mul_negi(mix_scale(P::sub(v[1], v[2]), K_SQRT3_2()));
      out[mix_slot(ob)] = P::add(v[0], t1);
      out[mix_slot(ob + Ns)] = P::add(t2, t3);
      out[mix_slot(ob + 2 * Ns)] = P::sub(t2, t3);
    } else {
      V acc = v[0];
#pragma unroll
      for (int r = 1; r < PO; ++r) acc = P::add(acc, v[r]);
      out[mix_slot(ob)] = acc;
#pragma unroll 1
      for (int q = 1; q < PO; ++q) {
        acc = v[0];
#pragma unroll
        for (int r = 1; r < PO; ++r) acc = P::add(acc, P::mul_tw(v[r], P::expand(roots[((q * r) % PO) * RQ])));
        out[mix_slot(ob + q * Ns)] = acc;
      }
    }
  }
}

// Three CTAs per SM where shared memory allows (a 1536-element complex128
// tile takes 62 KiB with its tables): the register budget then holds every
// variant at 80 registers without spills, and 24 warps per SM hide more of
// the latency and barrier stalls than 16.
constexpr int kMixmMinBlocks = 3;

// Dynamic shared memory: two padded buffers of C*R values, then R roots.
template <class P, int M>
__global__ void __launch_bounds__(kMixThreads, kMixmMinBlocks) efft_pass_mixm(void* __restrict__ data, const MixArgs a) {
  typedef typename P::V V;
  constexpr int KIND = MID;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float4 vtab[kMixPerThread * 32];
  __shared__ float4 wtab[kMixThreads];  // W_t of each thread, kept out of registers across the stages
  const int b = a.log2b, lc = a.log2C, ls = a.log2s;
  const int R = M << b, C = 1 << lc, CR = R << lc, CRP = CR + CR / 16;
  V* in = reinterpret_cast<V*>(smem_raw);
  V* out = in + CRP;
  float4* roots = reinterpret_cast<float4*>(out + CRP);

  int D = 0;
  if (P::kElemBytes == 16) D = (int)__ldg(state) - 127;
  const uint64_t runit = a.N / (uint64_t)R, tw_unit = a.N / a.L;
  for (int j = threadIdx.x; j < R; j += kMixThreads) roots[j] = twiddle_mix(a, (uint64_t)j * runit);

  // columns jcol0 .. jcol0 + C - 1, all in block jcol0 / s (C divides s)
  const uint64_t jcol0 = (uint64_t)blockIdx.x << lc;
  const uint64_t m0 = jcol0 & ((1ull << ls) - 1ull);
  const uint64_t base0 = (jcol0 >> ls) * a.L + m0;
  const int c = threadIdx.x & (C - 1), r0 = threadIdx.x >> lc, RS = kMixThreads >> lc;
  // pass twiddle factors: V_c[i] = W(m_c RS i), W_t = W(m_c r0)
  if (threadIdx.x < kMixPerThread * C) {
    const int i = threadIdx.x >> lc;
    if (i * RS < R) vtab[threadIdx.x] = twiddle_mix(a, (m0 + c) * (uint64_t)(i * RS) * tw_unit);
  }
  wtab[threadIdx.x] = (r0 < R) ? twiddle_mix(a, (m0 + c) * (uint64_t)r0 * tw_unit) : make_float4(1.f, 0.f, 0.f, 0.f);

  {
    V x[kMixPerThread];
#pragma unroll
    for (int i = 0; i < kMixPerThread; ++i) {
      const int r = r0 + i * RS;
      if (r < R) x[i] = Mem<P, KIND>::load(data, base0 + c + ((uint64_t)r << ls), D, 0u);
    }
#pragma unroll
    for (int i = 0; i < kMixPerThread; ++i) {
      const int r = r0 + i * RS;
      if (r < R) in[mix_slot(c * R + r)] = x[i];
    }
  }
  __syncthreads();

  int s0 = 0;
  for (; s0 + 3 <= b; s0 += 3) {
    mixm_pow2_stage<P, M, 3>(in, out, b, lc, s0, roots);
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
  }
  if (b > s0) {
    switch (b - s0) {
      case 1: mixm_pow2_stage<P, M, 1>(in, out, b, lc, s0, roots); break;
      case 2: mixm_pow2_stage<P, M, 2>(in, out, b, lc, s0, roots); break;
      default: mixm_pow2_stage<P, M, 3>(in, out, b, lc, s0, roots); break;
    }
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
  }
  constexpr int P0 = MixOdd<M>::p0, P1 = MixOdd<M>::p1;
  mixm_odd_stage<P, M, P0, 1>(in, out, b, lc, roots);
  __syncthreads();
  {
    V* t = in;
    in = out;
    out = t;
  }
  if constexpr (P1 > 1) {
    mixm_odd_stage<P, M, P1, P0>(in, out, b, lc, roots);
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
  }

  // epilogue: in[c*R + r] holds X[r] of column c
  const typename P::TW wt = P::expand(wtab[threadIdx.x]);
  const uint64_t base = (((uint64_t)blockIdx.x << lc) >> ls) * a.L + (((uint64_t)blockIdx.x << lc) & ((1ull << ls) - 1ull)) + c;
#pragma unroll
  for (int i = 0; i < kMixPerThread; ++i) {
    const int r = (threadIdx.x >> lc) + i * RS;
    if (r < R) {
      const V v = P::pass_tw(in[mix_slot(c * R + r)], wt, P::expand(vtab[i * C + c]));
      Mem<P, KIND>::store(data, base + ((uint64_t)r << ls), v, 0, 0u, false);
    }
  }
}

// ----------------------------------------------------------------------------
// Middle pass of N = 3 * 2^e with R = 3 * 2^b, b = 4..6 (R = 48, 96, 192),
// in two register stages and one shared-memory exchange (the Stockham kernel
// above exchanges every stage through shared memory):
//   R = P1 * 16, P1 = 3 * 2^(b-4); n = n2 + 16 n1, k = k1 + P1 k2;
//   stage A, thread n2 < 16 of its column: the P1-point DFT over
//     x[n2 + 16 n1] (a radix-3 butterfly over n1 = j, j + Q, j + 2Q,
//     Q = P1 / 3, times exp(-2*pi*i*j*q/P1), then radix-Q DIF in registers:
//     output q + 3 r in the register of bitrev(r)), times
//     exp(-2*pi*i*n2*k1/R), to shared memory at (k1, n2);
//   stage B, thread k1 < P1: the 16-point DIF over n2, output k1 + P1 k2,
//     the pass twiddle exp(-2*pi*i*m*k/L) = W(m k1) W(m P1 k2) (the first
//     per thread, the second per column from a table), stored.
// C = 16 columns per CTA, 256 threads (stage B uses 16 P1 of them); the R-th
// roots of unity come from the two-level table once per CTA.  Three CTAs per
// SM: at 85 registers the complex128 forms spill a few words, and the eight
// extra warps per SM still made the pass 5 % faster than two CTAs without
// spills.
// ----------------------------------------------------------------------------
constexpr int kM3Cols = 16;

template <class P, int P1>
__global__ void __launch_bounds__(kMixThreads, 3) efft_pass_m3(void* __restrict__ data, const MixArgs a) {
  typedef typename P::V V;
  constexpr int KIND = MID, C = kM3Cols, R = P1 * 16, Q = P1 / 3, LQ = (Q == 1) ? 0 : (Q == 2) ? 1 : 2;
  static_assert(P1 == 3 || P1 == 6 || P1 == 12, "R = 48, 96 or 192");
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  const uint32_t* state = a.state + (a.ptrs ? 4u * blockIdx.y : 0u);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);                     // [k1][n2][c], one pad slot per 16
  __shared__ float4 roots[R];                                 // exp(-2*pi*i*j/R)
  __shared__ float4 vtab[16 * C];                             // W(m_c P1 k2), [k2][c]
  auto slot = [](int k1, int n2, int c) {
    const int raw = ((k1 << 4) + n2) * C + c;
    return raw + (raw >> 4);
  };
  int D = 0;
  if (P::kElemBytes == 16) D = (int)__ldg(state) - 127;
  const uint64_t runit = a.N / (uint64_t)R, tw_unit = a.N / a.L;

  // columns jcol0 .. jcol0 + C - 1, all in block jcol0 / s (C divides s)
  const uint64_t jcol0 = (uint64_t)blockIdx.x * C;
  const uint64_t m0 = jcol0 & ((1ull << a.log2s) - 1ull);
  const uint64_t base0 = (jcol0 >> a.log2s) * a.L + m0;
  const int c = threadIdx.x & (C - 1), t = threadIdx.x >> 4;  // t: n2 in stage A, k1 in stage B

  // ---- stage A: thread n2 = t, the P1 rows n2 + 16 n1 of column c ----
  {
    // the tile's loads are issued first: they are in flight while the roots
    // and the pass twiddles are built and the CTA meets at the barrier
    V v[P1];
#pragma unroll
    for (int n1 = 0; n1 < P1; ++n1)
      v[n1] = Mem<P, KIND>::load(data, base0 + c + ((uint64_t)(t + 16 * n1) << a.log2s), D, 0u);
    for (int j = threadIdx.x; j < R; j += kMixThreads) roots[j] = twiddle_mix(a, (uint64_t)j * runit);
    {
      const int k2 = threadIdx.x >> 4, cc = threadIdx.x & (C - 1);
      vtab[k2 * C + cc] = twiddle_mix(a, (m0 + cc) * (uint64_t)(P1 * k2) * tw_unit);
    }
    __syncthreads();  // roots
    // radix 3 over (j, j + Q, j + 2Q), then exp(-2*pi*i*j*q/P1) = roots[16 j q]
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const V x0 = v[j], x1 = v[j + Q], x2 = v[j + 2 * Q];
      const V t1 = P::add(x1, x2);
      const V t2 = P::sub(x0, mix_scale(t1, df{0.5f, 0.f}));
      const V t3 = P::mul_negi(mix_scale(P::sub(x1, x2), K_SQRT3_2()));
      v[j] = P::add(x0, t1);
      v[j + Q] = P::add(t2, t3);
      v[j + 2 * Q] = P::sub(t2, t3);
      if (j > 0) {
        v[j + Q] = P::mul_tw(v[j + Q], P::expand(roots[16 * j]));
        v[j + 2 * Q] = P::mul_tw(v[j + 2 * Q], P::expand(roots[32 * j]));
      }
    }
    // radix-Q DIF of each third: register q Q + u holds output q + 3 bitrev(u)
    if constexpr (LQ > 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) dif_regs<P, LQ>(v + q * Q);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
      for (int u = 0; u < Q; ++u) {
        const int k1 = q + 3 * bitrev_c(u, LQ);
        V y = v[q * Q + u];
        if (k1 > 0 && t > 0) y = P::mul_tw(y, P::expand(roots[t * k1]));
        sm[slot(k1, t, c)] = y;
      }
    }
  }
  __syncthreads();

  // ---- stage B: thread k1 = t < P1, the 16 points n2 of column c ----
  if (t < P1) {
    V v[16];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) v[n2] = sm[slot(t, n2, c)];
    dif_regs<P, 4>(v);
    const typename P::TW wt = P::expand(twiddle_mix(a, (m0 + c) * (uint64_t)t * tw_unit));
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k2 = bitrev_c(u, 4);
      const int k = t + P1 * k2;
      const V y = P::pass_tw(v[u], wt, P::expand(vtab[k2 * C + c]));
      Mem<P, KIND>::store(data, base0 + c + ((uint64_t)k << a.log2s), y, 0, 0u, false);
    }
  }
}

// dynamic shared memory of efft_pass_m3: the padded C x R tile
constexpr int m3_smem_bytes(int R, int elem_bytes) {
  return (kM3Cols * R + kM3Cols * R / 16) * elem_bytes;
}

}  // namespace efft
