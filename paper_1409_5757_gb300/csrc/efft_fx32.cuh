// efft_fx32.cuh -- the complex64 pass kernel for radix R = 2^10 as two
// radix-32 stages (32 values per thread).  Included by efft_fx_f32.cu only.
#pragma once
#include <cuda.h>  // CUtensorMap (the struct only; no driver call is made here)
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/efft.h"
#include "efft_kernels.cuh"

namespace efft {

// cos / sin of pi/16 and 3*pi/16 as (hi, lo) float pairs (the exp(-2*pi*i*e/32)
// factors of the radix-32 butterflies; those of even e are the radix-16 ones).
__device__ __forceinline__ df K_C1_32() { return {0x1.f6297cp-1f, 0x1.feeb96p-26f}; }
__device__ __forceinline__ df K_S1_32() { return {0x1.8f8b84p-3f, -0x1.cb2cfap-30f}; }
__device__ __forceinline__ df K_C3_32() { return {0x1.a9b662p-1f, 0x1.21d434p-26f}; }
__device__ __forceinline__ df K_S3_32() { return {0x1.1c73b4p-1f, -0x1.9465cep-27f}; }

// x * exp(-2*pi*i*e/32), e = 0..15 (compile-time after unrolling).
template <class P>
__device__ __forceinline__ typename P::V tw32(int e, typename P::V x) {
  if ((e & 1) == 0) return tw16<P>(e >> 1, x);
  // exp(-2*pi*i*e/32) = cos(pi e/16) - i sin(pi e/16)
  switch (e) {
    case 1: return P::mul_const(x, K_C1_32(), P::negd(K_S1_32()));
    case 3: return P::mul_const(x, K_C3_32(), P::negd(K_S3_32()));
    case 5: return P::mul_const(x, K_S3_32(), P::negd(K_C3_32()));
    case 7: return P::mul_const(x, K_S1_32(), P::negd(K_C1_32()));
    case 9: return P::mul_const(x, P::negd(K_S1_32()), P::negd(K_C1_32()));
    case 11: return P::mul_const(x, P::negd(K_S3_32()), P::negd(K_C3_32()));
    case 13: return P::mul_const(x, P::negd(K_C3_32()), P::negd(K_S3_32()));
    default: return P::mul_const(x, P::negd(K_C1_32()), P::negd(K_S1_32()));
  }
}

// In-register radix-32 decimation in frequency (the butterfly pair of
// Eqs. 5-6 level by level); register u ends up holding output bitrev5(u).
template <class P>
__device__ __forceinline__ void dif32_regs(typename P::V* v) {
#pragma unroll
  for (int half = 16; half >= 1; half /= 2) {
#pragma unroll
    for (int blk = 0; blk < 32; blk += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        typename P::V a = v[blk + j], b = v[blk + j + half];
        v[blk + j] = P::add(a, b);
        v[blk + j + half] = tw32<P>(j * (16 / half), P::sub(a, b));
      }
    }
  }
}

// ----------------------------------------------------------------------------
// The pass of efft_pass_fx for R = 1024 = 32 * 32 rows and C = 2^LC columns
// (complex64): with n = t + 32 j (t, j < 32) and output k = q + 32 k2,
//   stage 0 (thread t of its column):  Y_t[q] = sum_j x[t + 32 j] W32^(j q),
//                                      times W1024^(t q), to shared memory;
//   stage 1 (thread q of its column):  X[q + 32 k2] = sum_t Y_t[q] W32^(t k2).
// One shared-memory exchange per pass (the radix-16 form 16 * 16 * 4 needs
// two, and a third to reorder the last pass's output): the L1 data pipe,
// not the FP32 pipe, bounds the complex64 passes.
//  - strided passes (FIRST, MID): C adjacent columns in adjacent threads
//    (row-major shared memory, raw = p*C + c, eight pad slots per 256 raw:
//    stage-0 writes and stage-1 reads both conflict-free for C = 8 and 16);
//    the first pass of a large array takes C = 16 (128 bytes per row
//    segment, 512 threads, one CTA per SM);
//  - last pass: a warp holds one column, lanes walk t (loads of 256
//    contiguous bytes), raw = c*R + p with one pad slot per 32, and the
//    stage-1 outputs k = q + 32 k2 of the 32 lanes are contiguous, so the
//    result goes straight to global memory.  Stage-0 twiddles then come from
//    a shared copy of the 1024-th roots (root k at k + k/8).
// The pass twiddle exp(-2*pi*i*m*k/L) = W(m q) * W(m 32 k2): the first per
// thread, the second per column in shared memory, as in efft_pass_fx.
// ----------------------------------------------------------------------------
template <int KIND, int LC, int MINB = 2>
__global__ void __launch_bounds__(32 << LC, MINB) efft_pass_fx32(void* __restrict__ data, const PassArgs a) {
  typedef PolicyF32 P;
  typedef float2 V;
  if (a.ptrs) data = a.ptrs[blockIdx.y];
  constexpr int R = 1024, C = 1 << LC, NT = 32 * C;
  constexpr bool STRIDED = (KIND == FIRST || KIND == MID);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  __shared__ float4 vtw[STRIDED ? 32 * C : 1];
  __shared__ float4 wroot[STRIDED ? 1 : R + R / 8];
  auto slot = [](int p, int col) {
    const int raw = STRIDED ? (p << LC) + col : (col << 10) + p;
    return STRIDED ? raw + ((raw >> 8) << 3) : raw + (raw >> 5);
  };

  const int tid = threadIdx.x;
  const int c = STRIDED ? (tid & (C - 1)) : (tid >> 5);
  const int t = STRIDED ? (tid >> LC) : (tid & 31);
  const uint64_t jcol = (uint64_t)blockIdx.x * C + c;
  uint64_t m = 0, colbase, step;
  if (KIND == FIRST) {
    step = (uint64_t)a.s_odd << a.log2s;
    m = jcol;
    colbase = jcol;
  } else if (STRIDED) {
    step = 1ull << a.log2s;
    m = jcol & (step - 1);
    colbase = ((jcol >> a.log2s) << a.log2L) + m;
  } else {
    step = 1;
    colbase = jcol << 10;
  }
  const int Dout = a.out_shift;

  // pass twiddle factors: V_c[k2] = W(m_c 32 k2) ([k2][c]), W_t = W(m t)
  float4 wt = make_float4(1.f, 0.f, 0.f, 0.f);
  if (STRIDED) {
    const int sh = (KIND == FIRST) ? 0 : a.log2N - a.log2L;
    {
      const int cc = tid & (C - 1), k2 = tid >> LC;  // NT = 32 C entries, one per thread
      const uint64_t mc = ((uint64_t)blockIdx.x * C + cc) & (KIND == FIRST ? ~0ull : step - 1);
      vtw[k2 * C + cc] = twiddle_N(a, (mc * (uint64_t)(32 * k2)) << sh);
    }
    wt = twiddle_N(a, (m * (uint64_t)t) << sh);
  } else {
    for (int k = tid; k < R; k += NT) wroot[k + (k >> 3)] = __ldg(a.w2048 + 2 * k);
  }

  V v[32];
  // ---- stage 0: rows t + 32 j straight from global memory ----
  {
    const uint64_t b0 = colbase + (uint64_t)t * step, sj = 32ull * step;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = Mem<P, KIND>::load(data, b0 + (uint64_t)j * sj, 0, a.conj_in);
  }
  if (!STRIDED) __syncthreads();  // wroot
  dif32_regs<P>(v);
  // W1024^(t q), q = bitrev5(u), to position p = 32 q + t
#pragma unroll
  for (int u = 1; u < 32; ++u) {
    const int q = bitrev_c(u, 5);
    const int e = t * q;
    v[u] = P::mul_tw(v[u], STRIDED ? __ldg(a.w2048 + 2 * e) : wroot[e + (e >> 3)]);
  }
#pragma unroll
  for (int u = 0; u < 32; ++u) sm[slot(32 * bitrev_c(u, 5) + t, c)] = v[u];
  __syncthreads();

  // ---- stage 1: thread q = t reads positions 32 q + j, j < 32 ----
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = sm[slot(32 * t + j, c)];
  dif32_regs<P>(v);

  // ---- epilogue: register u holds X[q + 32 k2], k2 = bitrev5(u) ----
  if (STRIDED) {
    const P::TW w = wt;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int k2 = bitrev_c(u, 5);
      const int k = t + 32 * k2;
      v[u] = P::pass_tw(v[u], w, vtw[k2 * C + c]);
      const uint64_t off = (KIND == FIRST) ? ((uint64_t)(k * a.s_odd) << a.log2s) : ((uint64_t)k << a.log2s);
      Mem<P, KIND>::store(data, colbase + off, v[u], Dout, a.conj_out, false);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int k = t + 32 * bitrev_c(u, 5);
      Mem<P, KIND>::store(data, colbase + (uint64_t)k, v[u], Dout, a.conj_out, false);
    }
  }
}

// Dynamic shared memory of efft_pass_fx32 with 2^LC columns: 1024 * 2^LC
// values plus one pad slot per 32.
constexpr int fx32_smem_bytes(int LC) { return ((1024 << LC) + (1024 << LC) / 32) * 8; }

// ----------------------------------------------------------------------------
// The wide complex64 first pass of 2^10 rows (the kernel above with C = 16,
// 512 threads, one CTA per SM), its tiles brought into shared memory by the
// tensor-memory accelerator.  The pass's columns j < s (s = N / 1024) with
// rows r < 1024 at element j + r s are the 2-D tensor [1024][s] of 8-byte
// elements; a tile is its 16 x 1024 box, four TMA copies of 16 x 256 (128
// bytes per row, so the column coordinate, a multiple of 16, is 128-byte
// aligned), completed on one mbarrier in shared memory.  The CTA is
// persistent: as soon as every thread has read the stage-1 inputs the
// buffer is free, and one thread issues the copies of its next tile, which
// land while stage 1, the pass twiddle and the stores of this tile run.
// Stage 0 reads the dense box (bank-conflict free: a warp's 32 lanes read
// two 128-byte rows), the exchange uses the padded layout of the kernel
// above.  Same arithmetic, same results as efft_pass_fx32<FIRST, 4>.
//
// The mbarrier wait is bounded (kTmaSpinLimit polls of try_wait): on expiry
// the CTA records EFFT_ERR_TIMEOUT in word 3 of the execute's state (read by
// efft_execute_check), waits once more, bounded, for the copies it issued,
// and returns.  a.inject_timeout (host-side fault injection) arms the
// barrier without issuing copies and polls only 1024 times.
// ----------------------------------------------------------------------------
constexpr uint32_t kTmaSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase `parity` of `bar`; true when it completed
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t n = 0; n < limit; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// generic-proxy accesses of shared memory before async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int LC>
__global__ void __launch_bounds__(32 << LC, 1)
efft_pass_fx32_tma(void* __restrict__ data, const PassArgs a, const __grid_constant__ CUtensorMap tmap) {
  typedef PolicyF32 P;
  typedef float2 V;
  constexpr int R = 1024, C = 1 << LC, TILE_BYTES = R * C * 8, BOX_ROWS = 256;
  static_assert(C * 8 == 128, "a tile row is one 128-byte box row");
  // the copies' destination is aligned up to 1024 bytes (the dynamic
  // allocation carries that much slack)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* const tile_base =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  V* sm = reinterpret_cast<V*>(tile_base);
  __shared__ float4 vtw[32 * C];
  __shared__ float4 wroot[R + R / 8];  // the 1024-th roots, root k at k + k/8
  __shared__ __align__(8) uint64_t bar;
  auto slot = [](int p, int col) {
    const int raw = (p << LC) + col;
    return raw + ((raw >> 8) << 3);
  };
  const int tid = threadIdx.x;
  const int c = tid & (C - 1);
  const int t = tid >> LC;
  const uint32_t limit = a.inject_timeout ? 1024u : kTmaSpinLimit;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  for (int k = tid; k < R; k += blockDim.x) wroot[k + (k >> 3)] = __ldg(a.w2048 + 2 * k);
  __syncthreads();

  // thread 0: arm the barrier with the tile's bytes and issue its copies
  auto issue = [&](uint64_t tl) {
    fence_proxy_async_smem();
    mbar_expect_tx(&bar, TILE_BYTES);
    if (!a.inject_timeout)
#pragma unroll
      for (int q = 0; q < R / BOX_ROWS; ++q)
        tma_load_2d(tile_base + q * BOX_ROWS * C * 8, &tmap, (int)(tl * C), q * BOX_ROWS, &bar);
  };
  uint64_t tile = blockIdx.x;
  uint32_t phase = 0;
  bool failed = false;
  if (tid == 0 && tile < a.ntiles) issue(tile);

  for (; tile < a.ntiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile's epilogue no longer reads vtw
    const uint64_t jcol = tile * C + c, m = jcol;
    {
      const int cc = tid & (C - 1), k2 = tid >> LC;
      vtw[k2 * C + cc] = twiddle_N(a, (tile * C + cc) * (uint64_t)(32 * k2));
    }
    const float4 wt = twiddle_N(a, m * (uint64_t)t);

    failed = !mbar_wait_bounded(&bar, phase, limit);
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    phase ^= 1u;

    V v[32];
    // ---- stage 0: rows t + 32 j of the dense box ----
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      v[j] = sm[((t + 32 * j) << LC) + c];
      if (a.conj_in) v[j].y = -v[j].y;
    }
    __syncthreads();  // the dense box is read before the exchange overwrites it
    dif32_regs<P>(v);
#pragma unroll
    for (int u = 1; u < 32; ++u) {
      const int e = t * bitrev_c(u, 5);
      v[u] = P::mul_tw(v[u], wroot[e + (e >> 3)]);
    }
#pragma unroll
    for (int u = 0; u < 32; ++u) sm[slot(32 * bitrev_c(u, 5) + t, c)] = v[u];
    __syncthreads();

    // ---- stage 1: thread q = t reads positions 32 q + j ----
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = sm[slot(32 * t + j, c)];
    __syncthreads();  // every stage-1 read is done: the buffer takes the next tile
    if (tid == 0 && tile + gridDim.x < a.ntiles) issue(tile + gridDim.x);
    dif32_regs<P>(v);

    // ---- epilogue: register u holds X[q + 32 k2], k2 = bitrev5(u) ----
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int k2 = bitrev_c(u, 5);
      const int k = t + 32 * k2;
      v[u] = P::pass_tw(v[u], wt, vtw[k2 * C + c]);
      Mem<P, FIRST>::store(data, jcol + ((uint64_t)k << a.log2s), v[u], 0, a.conj_out, false);
    }
  }
  if (failed) {
    if (tid == 0 && a.state) atomicOr(const_cast<uint32_t*>(a.state) + 3, (uint32_t)EFFT_ERR_TIMEOUT);
    // the copies this CTA issued must land before its shared memory is reused
    mbar_wait_bounded(&bar, phase, limit);
  }
}

constexpr int fx32_tma_smem_bytes() { return fx32_smem_bytes(4) + 1024; }

// ----------------------------------------------------------------------------
// The wide complex64 middle pass of 2^11 rows (radix-16 stages, 8 columns,
// 1024 threads, one CTA per SM; efft_pass_fx<PolicyF32, MID, 11, 3, 1>) as a
// persistent kernel fed by TMA copies.  The pass works on blocks of L = R s
// elements (s = 2^log2s, the column stride); block b's columns m < s with
// rows r < R at element b L + m + r s are the 3-D tensor [N/L][R][s] of
// 8-byte elements, and a tile (8 adjacent columns of one block) is R / 256
// boxes of 8 x 256 x 1 (64 bytes per row; the column coordinate, a multiple
// of 8, is 64-byte aligned).  Everything else as in efft_pass_fx32_tma:
// the next tile's copies are issued once the last stage has read its
// inputs, stage 0 reads the dense box, a barrier separates those reads from
// the padded exchange layout, and the mbarrier wait is bounded, its expiry
// recorded in word 3 of the execute's state.  Same arithmetic, same results
// as the kernel that loads its own tiles.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <int LR, int LC>
__global__ void __launch_bounds__(1 << (LR + LC - 4), 1)
efft_pass_mid_tma_f32(void* __restrict__ data, const PassArgs a, const __grid_constant__ CUtensorMap tmap) {
  typedef PolicyF32 P;
  typedef P::V V;
  constexpr int R = 1 << LR, C = 1 << LC, TPC = R >> 4;
  constexpr int NFULL = LR / 4, REM = LR % 4, NST = NFULL + (REM ? 1 : 0);
  constexpr int NMID = NST - 2;
  constexpr int BOX_ROWS = 256, TILE_BYTES = R * C * 8;
  static_assert(R % BOX_ROWS == 0 && (C * 8) % 16 == 0, "box shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* const tile_base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  V* sm = reinterpret_cast<V*>(tile_base);
  __shared__ P::TW vtw[16 * C];
  __shared__ float4 wroot[2048 + 256];  // the 2048-th roots, root k at k + k/8
  __shared__ __align__(8) uint64_t bar;
  auto slot = [](int p, int col) {
    const int raw = (p << LC) + col;
    return raw + (raw >> 4);
  };
  const int tid = threadIdx.x;
  const int c = tid & (C - 1);
  const int t = tid >> LC;
  const int kt = digit_rev_c(t << 4, LR);
  const int sb0 = slot(t, c);
  const int sh = a.log2N - a.log2L;
  const uint64_t smask = (1ull << a.log2s) - 1ull;
  const uint32_t limit = a.inject_timeout ? 1024u : kTmaSpinLimit;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  for (int k = tid; k < 2048; k += blockDim.x) wroot[k + (k >> 3)] = __ldg(a.w2048 + k);
  __syncthreads();
  auto issue = [&](uint64_t tl) {
    const uint64_t j0 = tl << LC;
    const int blk = (int)(j0 >> a.log2s), m0 = (int)(j0 & smask);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar, TILE_BYTES);
    if (!a.inject_timeout)
#pragma unroll
      for (int q = 0; q < R / BOX_ROWS; ++q) tma_load_3d(tile_base + q * BOX_ROWS * C * 8, &tmap, m0, q * BOX_ROWS, blk, &bar);
  };
  uint64_t tile = blockIdx.x;
  uint32_t phase = 0;
  bool failed = false;
  if (tid == 0 && tile < a.ntiles) issue(tile);

  for (; tile < a.ntiles; tile += gridDim.x) {
    const uint64_t jcol = (tile << LC) + c;
    const uint64_t m = jcol & smask;
    const uint64_t colbase = ((jcol >> a.log2s) << a.log2L) + m;
    __syncthreads();  // the previous tile's epilogue no longer reads vtw
    if (tid < 16 * C) {
      const int cc = tid >> 4, u = tid & 15;
      const uint64_t mc = ((tile << LC) + cc) & smask;
      const int kc = digit_rev_c(last_pos_c(u, REM), LR);
      vtw[u * C + cc] = P::expand(twiddle_N(a, (mc * (uint64_t)kc) << sh));
    }
    const P::TW wt = P::expand(twiddle_N(a, (m * (uint64_t)kt) << sh));

    failed = !mbar_wait_bounded(&bar, phase, limit);
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    phase ^= 1u;

    V v[16];
    // ---- stage 0: rows t + TPC*j of the dense box ----
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = sm[((t + TPC * j) << LC) + c];
    __syncthreads();  // the dense box is read before the exchange overwrites it
    dif_regs<P, 4>(v);
#pragma unroll
    for (int u = 1; u < 16; ++u) {
      const int e = (t * bitrev_c(u, 4)) << (11 - LR);
      v[u] = P::mul_tw(v[u], wroot[e + (e >> 3)]);
    }
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
      for (int u = 1; u < 16; ++u) {
        const int e = (i * bitrev_c(u, 4)) << (11 - log2l);
        v[u] = P::mul_tw(v[u], wroot[e + (e >> 3)]);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) sm[sb + pad_off(bitrev_c(u, 4) * gstep)] = v[u];
      __syncthreads();
    }

    // ---- last stage; then the buffer takes the next tile ----
    {
      const int sb = slot(t << 4, c);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = sm[sb + pad_off(j * C)];
    }
    __syncthreads();
    if (tid == 0 && tile + gridDim.x < a.ntiles) issue(tile + gridDim.x);
    if (REM == 0) dif_regs<P, 4>(v);
    else dif_groups<P, (REM == 0 ? 4 : REM)>(v);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = kt | digit_rev_c(last_pos_c(u, REM), LR);
      v[u] = P::pass_tw(v[u], wt, vtw[u * C + c]);
      Mem<P, MID>::store(data, colbase + ((uint64_t)k << a.log2s), v[u], 0, 0u, false);
    }
  }
  if (failed) {
    if (tid == 0 && a.state) atomicOr(const_cast<uint32_t*>(a.state) + 3, (uint32_t)EFFT_ERR_TIMEOUT);
    mbar_wait_bounded(&bar, phase, limit);
  }
}

// padded 16384-element tile of 8-byte elements plus alignment slack
constexpr int mid_tma_smem_bytes() { return ((1 << 14) + (1 << 14) / 16 + 1) * 8 + 1024; }

}  // namespace efft
