// efft_arith.cuh -- element arithmetic for the pass kernels.
//
// Two policies share one kernel body:
//   DF  : complex128 data.  GB300 issues FP64 FMA at ~1/70 of the FP32 rate,
//         so the butterflies run in double-float ("df") arithmetic: a real
//         value is an unevaluated pair h + l of FP32 numbers; sums use Knuth's
//         TwoSum and products the FMA-based TwoProd, giving ~48-bit
//         significands.  Conversion to/from the binary64 array is pure
//         integer bit manipulation (no FP64 instruction on the data path).
//   F32 : complex64 data, FP32 butterflies with twiddles stored as (hi, lo)
//         FP32 pairs generated from FP64, applied as a compensated product.
//
// Twiddle factors (Eq. 4 of Sec. 2.2: exp(-2*pi*i*k/N)) are always float4
// {re.h, re.l, im.h, im.l}.  All kernels compute the sign = -1 transform;
// sign = +1 is obtained by conjugating input and output.
//
// Every operation is written with explicit __f*_rn intrinsics so that the
// compiler cannot contract or reassociate the error-free transformations.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace efft {

// ---------------------------------------------------------------------------
// double-float scalars
// ---------------------------------------------------------------------------
struct df { float h, l; };
struct __align__(16) cdf { df re, im; };  // 16-byte aligned: one 128-bit access

__device__ __forceinline__ df df_add(df a, df b) {
  // TwoSum(a.h, b.h) (Knuth), low parts added without renormalisation.
  float s = __fadd_rn(a.h, b.h);
  float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return {s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}
__device__ __forceinline__ df df_sub(df a, df b) {
  float s = __fsub_rn(a.h, b.h);
  float bb = __fsub_rn(s, a.h);
  float e = __fsub_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fadd_rn(b.h, bb));
  return {s, __fadd_rn(__fsub_rn(a.l, b.l), e)};
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
// a * c for a constant c = c.h + c.l (TwoProd on the high parts).
__device__ __forceinline__ df df_mulc(df a, df c) {
  float p = __fmul_rn(a.h, c.h);
  float e = __fmaf_rn(a.h, c.h, -p);
  e = __fmaf_rn(a.h, c.l, e);
  e = __fmaf_rn(a.l, c.h, e);
  return {p, e};
}
// Fast2Sum renormalisation (|l| <= ulp(h)/2 afterwards).
__device__ __forceinline__ df df_norm(df a) {
  float s = __fadd_rn(a.h, a.l);
  return {s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

// a * w, w a normalised df twiddle {re.h, re.l, im.h, im.l}.
__device__ __forceinline__ cdf cdf_mul(cdf a, float4 w) {
  cdf r;
  {
    float p1 = __fmul_rn(a.re.h, w.x), e1 = __fmaf_rn(a.re.h, w.x, -p1);
    float p2 = __fmul_rn(a.im.h, w.z), e2 = __fmaf_rn(a.im.h, w.z, -p2);
    float s = __fsub_rn(p1, p2);
    float bb = __fsub_rn(s, p1);
    float t = __fsub_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fadd_rn(p2, bb));
    float lo = __fadd_rn(__fsub_rn(e1, e2), t);
    lo = __fmaf_rn(a.re.h, w.y, lo);
    lo = __fmaf_rn(a.re.l, w.x, lo);
    lo = __fmaf_rn(-a.im.h, w.w, lo);
    lo = __fmaf_rn(-a.im.l, w.z, lo);
    r.re = {s, lo};
  }
  {
    float p3 = __fmul_rn(a.re.h, w.z), e3 = __fmaf_rn(a.re.h, w.z, -p3);
    float p4 = __fmul_rn(a.im.h, w.x), e4 = __fmaf_rn(a.im.h, w.x, -p4);
    float s = __fadd_rn(p3, p4);
    float bb = __fsub_rn(s, p3);
    float t = __fadd_rn(__fsub_rn(p3, __fsub_rn(s, bb)), __fsub_rn(p4, bb));
    float lo = __fadd_rn(__fadd_rn(e3, e4), t);
    lo = __fmaf_rn(a.re.h, w.w, lo);
    lo = __fmaf_rn(a.re.l, w.z, lo);
    lo = __fmaf_rn(a.im.h, w.y, lo);
    lo = __fmaf_rn(a.im.l, w.x, lo);
    r.im = {s, lo};
  }
  return r;
}

// Product of two normalised df twiddles (two-level table lookup), normalised.
__device__ __forceinline__ float4 tw_mul(float4 a, float4 b) {
  cdf x{{a.x, a.y}, {a.z, a.w}};
  cdf y = cdf_mul(x, b);
  df re = df_norm(y.re), im = df_norm(y.im);
  return make_float4(re.h, re.l, im.h, im.l);
}

// cos(pi/8), sin(pi/8), cos(pi/4) as float pairs (hi = RN(v), lo = RN(v - hi)).
__device__ __forceinline__ df K_C1() { return {0.92387950420379638671875f, 2.830748968563057132996618747711181640625e-08f}; }
__device__ __forceinline__ df K_S1() { return {0.3826834261417388916015625f, 6.223350723644216486718505620956420898438e-09f}; }
__device__ __forceinline__ df K_R() { return {0.707106769084930419921875f, 1.21016174858823433169163763523101806640625e-08f}; }

// ---------------------------------------------------------------------------
// Policies
// ---------------------------------------------------------------------------
struct PolicyDF {
  typedef cdf V;
  typedef float4 TW;
  static constexpr int kElemBytes = 16;
  static __device__ __forceinline__ TW expand(float4 w) { return w; }
  static __device__ __forceinline__ TW int_tw(const float4* w, const float4*, uint32_t i) { return __ldg(w + i); }
  static __device__ __forceinline__ V pass_tw(V v, const TW& wt, const TW& vc) { return cdf_mul(v, tw_mul(wt, vc)); }
  static __device__ __forceinline__ V add(V a, V b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
  static __device__ __forceinline__ V sub(V a, V b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
  static __device__ __forceinline__ V mul_tw(V a, float4 w) { return cdf_mul(a, w); }
  static __device__ __forceinline__ V mul_const(V a, df wr, df wi) {
    return cdf_mul(a, make_float4(wr.h, wr.l, wi.h, wi.l));
  }
  // (a + ib) * r(1 - i) = r(a + b) + i r(b - a)
  static __device__ __forceinline__ V mul_w8(V x) {
    df r = K_R();
    return {df_mulc(df_add(x.re, x.im), r), df_mulc(df_sub(x.im, x.re), r)};
  }
  // (a + ib) * r(-1 - i) = r(b - a) - i r(a + b)
  static __device__ __forceinline__ V mul_w8_3(V x) {
    df r = K_R();
    return {df_mulc(df_sub(x.im, x.re), r), df_neg(df_mulc(df_add(x.re, x.im), r))};
  }
  static __device__ __forceinline__ V mul_negi(V x) { return {x.im, df_neg(x.re)}; }
  static __device__ __forceinline__ df C1() { return K_C1(); }
  static __device__ __forceinline__ df S1() { return K_S1(); }
  static __device__ __forceinline__ df negd(df a) { return df_neg(a); }
};

// Packed FP32x2 (sm_100+): one instruction, two FP32 operations.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  unsigned long long ua = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long ub = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long ud;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
  return *reinterpret_cast<float2*>(&ud);
}
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

struct PolicyF32 {
  typedef float2 V;
  typedef float4 TW;
  static constexpr int kElemBytes = 8;
  static __device__ __forceinline__ TW expand(float4 w) { return w; }
  static __device__ __forceinline__ TW int_tw(const float4* w, const float4*, uint32_t i) { return __ldg(w + i); }
  // complex add / subtract as one packed instruction each
  static __device__ __forceinline__ V add(V a, V b) { return f2add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return f2sub(a, b); }
  // compensated product: x*w = x*w_lo + x*w_hi, the lo part first
  static __device__ __forceinline__ V mul_tw(V a, float4 w) {
    float re = __fmaf_rn(-a.y, w.w, __fmul_rn(a.x, w.y));
    re = __fmaf_rn(a.x, w.x, re);
    re = __fmaf_rn(-a.y, w.z, re);
    float im = __fmaf_rn(a.y, w.y, __fmul_rn(a.x, w.w));
    im = __fmaf_rn(a.x, w.z, im);
    im = __fmaf_rn(a.y, w.x, im);
    return make_float2(re, im);
  }
  static __device__ __forceinline__ V mul_const(V a, df wr, df wi) {
    return mul_tw(a, make_float4(wr.h, wr.l, wi.h, wi.l));
  }
  static __device__ __forceinline__ float mulr(float v) {
    df r = K_R();
    return __fmaf_rn(v, r.h, __fmul_rn(v, r.l));
  }
  static __device__ __forceinline__ V mul_w8(V x) {
    return make_float2(mulr(__fadd_rn(x.x, x.y)), mulr(__fsub_rn(x.y, x.x)));
  }
  static __device__ __forceinline__ V mul_w8_3(V x) {
    return make_float2(mulr(__fsub_rn(x.y, x.x)), -mulr(__fadd_rn(x.x, x.y)));
  }
  static __device__ __forceinline__ V mul_negi(V x) { return make_float2(x.y, -x.x); }
  static __device__ __forceinline__ df C1() { return K_C1(); }
  static __device__ __forceinline__ df S1() { return K_S1(); }
  static __device__ __forceinline__ df negd(df a) { return df_neg(a); }
  // the pass twiddle W_t * V_c applied as two compensated products (12
  // operations, against 38 for forming W_t * V_c in double-float first)
  static __device__ __forceinline__ V pass_tw(V v, const TW& wt, const TW& vc) { return mul_tw(mul_tw(v, wt), vc); }
};

// ---------------------------------------------------------------------------
// Packed double-float complex ("DF2"): sm_100+ FP32x2 instructions carry the
// real and imaginary halves together.  h = (re.h, im.h), l = (re.l, im.l).
// A packed instruction does two FP32 operations in one issue slot (measured:
// same FP32 throughput as scalar, half the instructions).
// ---------------------------------------------------------------------------
struct __align__(16) cdf2 { float2 h, l; };
// expanded twiddle w = wr + i wi for the packed multiply:
// a = (wr, wr), b = (-wi, wi), al / bl the same for the low parts
struct __align__(16) tw2 { float2 a, b, al, bl; };


__device__ __forceinline__ cdf2 c2add(cdf2 a, cdf2 b) {
  float2 s = f2add(a.h, b.h);
  float2 bb = f2sub(s, a.h);
  float2 e = f2add(f2sub(a.h, f2sub(s, bb)), f2sub(b.h, bb));
  return {s, f2add(f2add(a.l, b.l), e)};
}
__device__ __forceinline__ cdf2 c2sub(cdf2 a, cdf2 b) {
  float2 s = f2sub(a.h, b.h);
  float2 bb = f2sub(s, a.h);
  float2 e = f2sub(f2sub(a.h, f2sub(s, bb)), f2add(b.h, bb));
  return {s, f2add(f2sub(a.l, b.l), e)};
}
// x * w (w expanded).  re = xr wr - xi wi, im = xi wr + xr wi:
// P = x.h (wr, wr), Q = swap(x.h) (-wi, wi), S = P + Q exactly split by TwoSum.
__device__ __forceinline__ cdf2 c2mul(cdf2 x, const tw2& w) {
  const float2 xs = make_float2(x.h.y, x.h.x);
  const float2 ls = make_float2(x.l.y, x.l.x);
  float2 P = f2mul(x.h, w.a);
  float2 Q = f2mul(xs, w.b);
  float2 E1 = f2fma(x.h, w.a, f2neg(P));
  float2 E2 = f2fma(xs, w.b, f2neg(Q));
  float2 S = f2add(P, Q);
  float2 bb = f2sub(S, P);
  float2 t = f2add(f2sub(P, f2sub(S, bb)), f2sub(Q, bb));
  float2 lo = f2add(f2add(E1, E2), t);
  lo = f2fma(x.h, w.al, lo);
  lo = f2fma(xs, w.bl, lo);
  lo = f2fma(x.l, w.a, lo);
  lo = f2fma(ls, w.b, lo);
  return {S, lo};
}
__device__ __forceinline__ tw2 tw_expand(float4 w) {  // natural {re.h, re.l, im.h, im.l}
  tw2 r;
  r.a = make_float2(w.x, w.x);
  r.b = make_float2(-w.z, w.z);
  r.al = make_float2(w.y, w.y);
  r.bl = make_float2(-w.w, w.w);
  return r;
}
__device__ __forceinline__ cdf2 c2negi(cdf2 x) {  // x * (-i) = (im, -re)
  return {make_float2(x.h.y, -x.h.x), make_float2(x.l.y, -x.l.x)};
}
// real df constant c times both halves
__device__ __forceinline__ cdf2 c2mulr(cdf2 x, df c) {
  const float2 ch = make_float2(c.h, c.h), cl = make_float2(c.l, c.l);
  float2 p = f2mul(x.h, ch);
  float2 e = f2fma(x.h, ch, f2neg(p));
  e = f2fma(x.h, cl, e);
  e = f2fma(x.l, ch, e);
  return {p, e};
}
__device__ __forceinline__ cdf2 c2norm(cdf2 x) {
  float2 s = f2add(x.h, x.l);
  return {s, f2sub(x.l, f2sub(s, x.h))};
}

struct PolicyDF2 {
  typedef cdf2 V;
  typedef tw2 TW;
  static constexpr int kElemBytes = 16;
  static __device__ __forceinline__ TW expand(float4 w) { return tw_expand(w); }
  // the natural 16-byte table (32 KiB, stays in L1), expanded in registers
  static __device__ __forceinline__ TW int_tw(const float4* w, const float4*, uint32_t i) {
    return tw_expand(__ldg(w + i));
  }
  static __device__ __forceinline__ V mul_tw(V a, const TW& w) { return c2mul(a, w); }
  // the pass twiddle W_t * V_c applied as two packed products
  static __device__ __forceinline__ V pass_tw(V v, const TW& wt, const TW& vc) { return c2mul(c2mul(v, wt), vc); }
  static __device__ __forceinline__ V add(V a, V b) { return c2add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return c2sub(a, b); }
  static __device__ __forceinline__ V mul_const(V a, df wr, df wi) {
    tw2 w;
    w.a = make_float2(wr.h, wr.h);
    w.b = make_float2(-wi.h, wi.h);
    w.al = make_float2(wr.l, wr.l);
    w.bl = make_float2(-wi.l, wi.l);
    return c2mul(a, w);
  }
  // (a + ib) r(1 - i) = r(a + b) + i r(b - a) = r * (x + x*(-i))
  static __device__ __forceinline__ V mul_w8(V x) { return c2mulr(c2add(x, c2negi(x)), K_R()); }
  // (a + ib) r(-1 - i) = -i * [(a + ib) r(1 - i)]
  static __device__ __forceinline__ V mul_w8_3(V x) { return c2negi(mul_w8(x)); }
  static __device__ __forceinline__ V mul_negi(V x) { return c2negi(x); }
  static __device__ __forceinline__ df C1() { return K_C1(); }
  static __device__ __forceinline__ df S1() { return K_S1(); }
  static __device__ __forceinline__ df negd(df a) { return df_neg(a); }
};

// x * exp(-2*pi*i*e/16) for e = 0..7 (compile-time after unrolling).
template <class P>
__device__ __forceinline__ typename P::V tw16(int e, typename P::V x) {
  switch (e) {
    case 0: return x;
    case 1: return P::mul_const(x, P::C1(), P::negd(P::S1()));
    case 2: return P::mul_w8(x);
    case 3: return P::mul_const(x, P::S1(), P::negd(P::C1()));
    case 4: return P::mul_negi(x);
    case 5: return P::mul_const(x, P::negd(P::S1()), P::negd(P::C1()));
    case 6: return P::mul_w8_3(x);
    default: return P::mul_const(x, P::negd(P::C1()), P::negd(P::S1()));
  }
}

// In-register decimation-in-frequency radix-2^LOG DFT on v[0 .. 2^LOG)
// (the butterfly pair of Eqs. 5-6 applied level by level, Gentleman-Sande
// order).  Input natural order; register u ends up holding output
// bitrev_LOG(u).  LOG <= 4.
template <class P, int LOG>
__device__ __forceinline__ void dif_regs(typename P::V* v) {
  constexpr int n = 1 << LOG;
#pragma unroll
  for (int half = n / 2; half >= 1; half /= 2) {
#pragma unroll
    for (int blk = 0; blk < n; blk += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        typename P::V a = v[blk + j], b = v[blk + j + half];
        v[blk + j] = P::add(a, b);
        v[blk + j + half] = tw16<P>(j * (8 / half), P::sub(a, b));
      }
    }
  }
}

__host__ __device__ __forceinline__ int bitrev_n(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}

}  // namespace efft
