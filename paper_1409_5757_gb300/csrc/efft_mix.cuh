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

}  // namespace efft
