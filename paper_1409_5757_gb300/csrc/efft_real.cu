// efft_real.cu -- real-data transforms in the perm layout of Eq. 3 (Sec. 2.1)
// with the in-place combination of mirrored pairs (Sec. 3.4).
//
// N reals x are viewed as N/2 complex values z[m] = x[2m] + i x[2m+1].  With
// Z the N/2-point DFT of z (sign -1) and W = exp(-2*pi*i/N), the even and odd
// half-length spectra of Eq. 4 are E_k = (Z_k + conj Z_{N/2-k})/2 and
// O_k = (Z_k - conj Z_{N/2-k})/(2i), and F_k = E_k + W^k O_k (the butterfly
// of Eqs. 5-6), F_{N/2-k} = conj(E_k - W^k O_k).  Writing A = Z_k + Q,
// B = Z_k - Q (Q = conj Z_{N/2-k}) and D = -i W^k B:
//     F_k = (A + D) / 2,   F_{N/2-k} = conj(A - D) / 2,
// so one kernel thread reads slots k and N/2-k and writes both back: the pair
// is combined in place.  Slot 0 holds Z_0 and receives (F_0, F_{N/2}).  Any
// even N: N = M * 2^e with the complex plan of N/2 = M * 2^(e-1) points; when
// N/2 is odd no slot pairs with itself.  The inverse runs the same step
// first, with conj(W), +i and without the 1/2, and then the conjugate-sign
// complex transform.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/efft.h"
#include "efft_host.h"
#include "efft_kernels.cuh"

using namespace efft;
using namespace efft::host;

namespace {

struct RealArgs {
  uint64_t nh;            // complex values: N/2
  int rtwB;               // low-table bits of the W table
  const float4* lo;       // exp(-2*pi*i*t/N), t < 2^rtwB
  const float4* hi;       // exp(-2*pi*i*(t << rtwB)/N)
  const uint32_t* state;  // complex128: max biased exponent (word 0) for the scale
  int inverse;            // 0: Z -> perm (forward); 1: perm -> Z (inverse)
  int grow;               // complex128: log2 bound of |values| / 2^(emax-1023)
  int out_shift;          // outputs multiplied by 2^-out_shift
};

// W^m (conj(W)^m for the inverse) for 0 < m <= N/4 from the two-level table.
__device__ __forceinline__ float4 w_of(const RealArgs& a, uint64_t m) {
  const uint32_t lo = (uint32_t)(m & ((1ull << a.rtwB) - 1ull));
  const uint32_t hi = (uint32_t)(m >> a.rtwB);
  float4 w = tw_mul(__ldg(a.hi + hi), __ldg(a.lo + lo));
  if (a.inverse) w = make_float4(w.x, w.y, -w.z, -w.w);  // conj(W)
  return w;
}

// complex64: FP32 with the compensated twiddle product of the pass kernels.
__global__ void __launch_bounds__(256) efft_real_pairs_f32(float2* __restrict__ z, const RealArgs a) {
  const uint64_t half = a.nh >> 1;
  const float sc = __uint_as_float((uint32_t)(127 - a.out_shift) << 23);
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= half;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t km = (k == 0) ? 0 : a.nh - k;
    const float2 zk = __ldcg(z + k);
    float2 p, q;
    if (k == 0) {
      // forward: Z_0 and its conjugate; inverse: F_0 and F_{N/2}, both real
      p = a.inverse ? make_float2(zk.x, 0.f) : zk;
      q = a.inverse ? make_float2(zk.y, 0.f) : make_float2(zk.x, -zk.y);
    } else {
      const float2 zm = __ldcg(z + km);
      p = zk;
      q = make_float2(zm.x, -zm.y);
    }
    const float2 A = PolicyF32::add(p, q), B = PolicyF32::sub(p, q);
    // D = -i W^k B (inverse +i conj(W)^k B): exactly -i B at k = 0, -B at
    // k = N/4 (N/2 even), else with W^k from the table
    float2 D;
    if (k == 0) {
      D = a.inverse ? make_float2(-B.y, B.x) : make_float2(B.y, -B.x);
    } else if (2 * k == a.nh) {
      D = make_float2(-B.x, -B.y);
    } else {
      const float2 wb = PolicyF32::mul_tw(B, w_of(a, k));
      D = a.inverse ? make_float2(-wb.y, wb.x) : make_float2(wb.y, -wb.x);
    }
    float2 x = PolicyF32::add(A, D), y = PolicyF32::sub(A, D);
    x = make_float2(__fmul_rn(x.x, sc), __fmul_rn(x.y, sc));
    y = make_float2(__fmul_rn(y.x, sc), __fmul_rn(-y.y, sc));  // conj
    if (k == 0) {
      // forward: (F_0, F_{N/2}) = (x.re, y.re); inverse: Z_0 = x
      z[0] = a.inverse ? x : make_float2(x.x, y.x);
    } else {
      z[k] = x;
      if (km != k) z[km] = y;
    }
  }
}

// complex128: double-float, the binary64 values converted with an exact
// power-of-two scale (the bound on |values| comes from the range scan).
__global__ void __launch_bounds__(256) efft_real_pairs_df(uint4* __restrict__ z, const RealArgs a) {
  const uint64_t half = a.nh >> 1;
  const uint32_t emax = __ldg(a.state);
  const bool nonfinite = (emax >= 0x7FFu);
  const int D = (int)emax + a.grow - 127;
  const int Dout = D - a.out_shift;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= half;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t km = (k == 0) ? 0 : a.nh - k;
    const uint4 uk = __ldcg(z + k);
    cdf2 p, q;
    {
      const df re = f64bits_to_df(uk.x, uk.y, D, 0u), im = f64bits_to_df(uk.z, uk.w, D, 0u);
      if (k == 0) {
        if (a.inverse) {
          p = cdf2{make_float2(re.h, 0.f), make_float2(re.l, 0.f)};
          q = cdf2{make_float2(im.h, 0.f), make_float2(im.l, 0.f)};
        } else {
          p = cdf2{make_float2(re.h, im.h), make_float2(re.l, im.l)};
          q = cdf2{make_float2(re.h, -im.h), make_float2(re.l, -im.l)};
        }
      } else {
        const uint4 um = __ldcg(z + km);
        const df mre = f64bits_to_df(um.x, um.y, D, 0u);
        const df mim = f64bits_to_df(um.z, um.w, D, 0x80000000u);  // conj
        p = cdf2{make_float2(re.h, im.h), make_float2(re.l, im.l)};
        q = cdf2{make_float2(mre.h, mim.h), make_float2(mre.l, mim.l)};
      }
    }
    const cdf2 A = c2add(p, q), B = c2sub(p, q);
    // D = -i W^k B (inverse +i conj(W)^k B): exactly -i B at k = 0, -B at
    // k = N/4 (N/2 even), else with W^k from the table
    cdf2 Dv;
    if (k == 0) {
      Dv = a.inverse ? c2negi(c2negi(c2negi(B))) : c2negi(B);
    } else if (2 * k == a.nh) {
      Dv = cdf2{f2neg(B.h), f2neg(B.l)};
    } else {
      const cdf2 wb = c2mul(B, tw_expand(w_of(a, k)));
      Dv = a.inverse ? c2negi(c2negi(c2negi(wb))) : c2negi(wb);
    }
    const cdf2 x = c2add(A, Dv), y = c2sub(A, Dv);
    uint4 ox, oy;
    df_to_f64bits(df{x.h.x, x.l.x}, Dout, 0u, ox.x, ox.y);
    df_to_f64bits(df{x.h.y, x.l.y}, Dout, 0u, ox.z, ox.w);
    df_to_f64bits(df{y.h.x, y.l.x}, Dout, 0u, oy.x, oy.y);
    df_to_f64bits(df{y.h.y, y.l.y}, Dout, 0x80000000u, oy.z, oy.w);  // conj
    if (nonfinite) ox = oy = make_uint4(0u, 0x7FF80000u, 0u, 0x7FF80000u);
    if (k == 0) {
      z[0] = a.inverse ? ox : make_uint4(ox.x, ox.y, oy.x, oy.y);
    } else {
      z[k] = ox;
      if (km != k) z[km] = oy;
    }
  }
}

int launch_pairs(efft_plan_s* p, void* data, const uint32_t* state, int grow, cudaStream_t st) {
  RealArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nh = p->n >> 1;
  a.rtwB = p->rtwB;
  a.lo = p->rtw_lo;
  a.hi = p->rtw_hi;
  a.state = state;
  a.inverse = (p->real == EFFT_REAL_INVERSE) ? 1 : 0;
  a.grow = grow;
  // forward: the 1/2 of the pair formula; normalised: a further 1/2 (the
  // complex plan contributes 2/N)
  a.out_shift = (a.inverse ? 0 : 1) + ((p->flags & EFFT_FLAG_NORMALIZE) ? 1 : 0);
  uint64_t blocks = ((a.nh >> 1) + 1 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  int rec = prof_begin(p, 7, st);
  if (p->dtype == EFFT_C128)
    efft_real_pairs_df<<<(unsigned)blocks, 256, 0, st>>>(static_cast<uint4*>(data), a);
  else
    efft_real_pairs_f32<<<(unsigned)blocks, 256, 0, st>>>(static_cast<float2*>(data), a);
  prof_end(p, rec, st);
  return cudaGetLastError() == cudaSuccess ? EFFT_OK : EFFT_ERR_LAUNCH;
}

}  // namespace

namespace efft {
namespace host {

// Forward: the complex transform, then the pairs (the scale bound: the
// complex output is at most (N/2) sqrt(2) times the largest input, or
// sqrt(2) times it when normalised by 2/N).  Inverse: a range scan of the
// perm array, the pairs (|A|, |D| <= 2 max|F|), then the complex transform.
// One state word serves the whole execute: the complex transform's range
// scan writes it and the pair kernel then reads it (forward), or the pair
// kernel reads the perm array's scan before the complex transform rescans.
int enqueue_real(efft_plan_s* p, void* data, uint32_t* state, cudaStream_t st) {
  if (fault_injected("launch")) return EFFT_ERR_LAUNCH;
  efft_plan_s* in = p->inner;
  const bool c128 = (p->dtype == EFFT_C128);
  if (p->real == EFFT_REAL_FORWARD) {
    int rc = enqueue_state(in, data, state, st);
    if (rc != EFFT_OK) return rc;
    const int grow = 2 + ((p->flags & EFFT_FLAG_NORMALIZE) ? 0 : in->log2n);
    if (c128 && in->log2n == 0) {
      // N = 2: the one-point complex transform launches nothing, so no scan ran
      int rec = prof_begin(p, 0, st);
      rc = launch_range_scan(data, 1, state, nullptr, 1, st);
      prof_end(p, rec, st);
      if (rc != EFFT_OK) return rc;
    }
    return launch_pairs(p, data, c128 ? state : nullptr, grow, st);
  }
  if (c128) {
    int rec = prof_begin(p, 0, st);
    const int rc = launch_range_scan(data, p->n >> 1, state, nullptr, 1, st);
    prof_end(p, rec, st);
    if (rc != EFFT_OK) return rc;
  }
  int rc = launch_pairs(p, data, c128 ? state : nullptr, 2, st);
  if (rc != EFFT_OK) return rc;
  return enqueue_state(in, data, state, st);
}

}  // namespace host
}  // namespace efft

extern "C" int efft_plan_create_real(efft_plan_t* out, uint64_t n, int precision, int direction,
                                     uint32_t flags) {
  if (!out) return EFFT_ERR_INVALID_PTR;
  *out = nullptr;
  if (n < 2 || (n & 1) != 0 || n > (1ull << (EFFT_MAX_LOG2N + 1)) || !valid_size(n >> 1))
    return EFFT_ERR_INVALID_SIZE;
  if (precision != EFFT_C64 && precision != EFFT_C128) return EFFT_ERR_INVALID_DTYPE;
  if (direction != EFFT_REAL_FORWARD && direction != EFFT_REAL_INVERSE) return EFFT_ERR_INVALID_SIGN;
  if (flags & ~(EFFT_FLAG_NORMALIZE | EFFT_FLAG_AUTOTUNE)) return EFFT_ERR_INVALID_FLAGS;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return EFFT_ERR_CUDA;
  }
  // the complex plan of N/2 points (same sign, same normalisation request)
  efft_plan_t inner = nullptr;
  int rc = efft_plan_create(&inner, n >> 1, precision, direction, flags);
  if (rc != EFFT_OK) return rc;
  efft_plan_s* p = new (std::nothrow) efft_plan_s();
  if (!p) {
    efft_plan_destroy(inner);
    return EFFT_ERR_ALLOC;
  }
  std::memset(p, 0, sizeof(*p));
  p->device = dev;
  p->n = n;
  p->log2n = ilog2_u64(n);
  p->dtype = precision;
  p->sign = direction;
  p->flags = flags;
  p->real = direction;
  p->inner = inner;
  // W table exp(-2*pi*i*m/N) for m < 2^em (>= N/2), two-level
  const int em = p->log2n - 1;  // log2n = ceil(log2 N)
  p->rtwB = (em + 1) / 2;
  const uint64_t nlo = 1ull << p->rtwB, nhi = 1ull << (em - p->rtwB);
  cudaStream_t st = nullptr;
  if (fault_injected("alloc") || cudaMalloc(&p->rtw_lo, nlo * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&p->rtw_hi, nhi * sizeof(float4)) != cudaSuccess)
    rc = EFFT_ERR_ALLOC;
  if (rc == EFFT_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = EFFT_ERR_CUDA;
  if (rc == EFFT_OK) rc = gen_table(p->rtw_lo, nlo, 1, n, st);
  if (rc == EFFT_OK) rc = gen_table(p->rtw_hi, nhi, nlo, n, st);
  if (rc == EFFT_OK) rc = ring_create(p, st);
  if (rc == EFFT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = EFFT_ERR_CUDA;
  if (st) cudaStreamDestroy(st);
  p->recs = new (std::nothrow) std::vector<efft_plan_s::Rec>();
  p->pool = new (std::nothrow) std::vector<cudaEvent_t>();
  if (rc == EFFT_OK && (!p->recs || !p->pool)) rc = EFFT_ERR_ALLOC;
  if (rc != EFFT_OK) {
    cudaGetLastError();
    free_plan_memory(p);  // also destroys the complex plan
    delete p;
    return rc;
  }
  p->table_bytes = (nlo + nhi) * sizeof(float4) + 16 * kStateRing;
  p->magic = kMagic;
  register_plan(p);
  *out = p;
  return EFFT_OK;
}
