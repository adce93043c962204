// efft_mix.cu -- launches of the mixed-radix pass kernel (efft_pass_mix in
// efft_mix.cuh) for transform lengths N = M * 2^e with M odd (the
// paper's size set N = M * 2^s, Sec. 2.1).  A translation unit of its own:
// the kernel is instantiated for every odd radix and compiles in parallel
// with the others.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/efft.h"
#include "efft_host.h"
#include "efft_kernels.cuh"
#include "efft_mix.cuh"

using namespace efft;
using namespace efft::host;

namespace {

static_assert(kMixTileC128 <= kMixThreads * kMixPerThread && kMixTileC64 <= kMixThreads * kMixPerThread,
              "a tile is loaded and stored in kMixPerThread elements per thread");

template <class P, int KIND>
void launch_mix_kind(const MixArgs& m, const Pass& ps, void* data, unsigned count, cudaStream_t st) {
  efft_pass_mix<P, KIND><<<dim3((unsigned)ps.grid, count), kMixThreads, ps.smem, st>>>(data, m);
}

// The middle pass with the odd factor fixed at compile time (efft_pass_mixm).
template <class P, int M>
void launch_mixm(const MixArgs& m, const Pass& ps, void* data, unsigned count, cudaStream_t st) {
  efft_pass_mixm<P, M><<<dim3((unsigned)ps.grid, count), kMixThreads, ps.smem, st>>>(data, m);
}

template <class P>
bool launch_mixm_odd(int odd, const MixArgs& m, const Pass& ps, void* data, unsigned count, cudaStream_t st) {
  switch (odd) {
    case 3: launch_mixm<P, 3>(m, ps, data, count, st); return true;
    case 5: launch_mixm<P, 5>(m, ps, data, count, st); return true;
    case 7: launch_mixm<P, 7>(m, ps, data, count, st); return true;
    case 9: launch_mixm<P, 9>(m, ps, data, count, st); return true;
    case 11: launch_mixm<P, 11>(m, ps, data, count, st); return true;
    case 13: launch_mixm<P, 13>(m, ps, data, count, st); return true;
    case 15: launch_mixm<P, 15>(m, ps, data, count, st); return true;
    default: return false;
  }
}

// The middle pass of N = 3 * 2^e with R = 3 * 2^b, b = 4..6, in two register
// stages (efft_pass_m3): 16 columns per CTA.
template <class P, int P1>
void launch_m3(const MixArgs& m, const efft_plan_s* p, void* data, unsigned count, cudaStream_t st) {
  const uint64_t tiles = p->n / (uint64_t)(P1 * 16) / (uint64_t)kM3Cols;
  efft_pass_m3<P, P1><<<dim3((unsigned)tiles, count), kMixThreads, m3_smem_bytes(P1 * 16, P::kElemBytes), st>>>(data, m);
}

template <class P>
bool launch_m3_b(int b, const MixArgs& m, const efft_plan_s* p, void* data, unsigned count, cudaStream_t st) {
  switch (b) {
    case 4: launch_m3<P, 3>(m, p, data, count, st); return true;
    case 5: launch_m3<P, 6>(m, p, data, count, st); return true;
    case 6: launch_m3<P, 12>(m, p, data, count, st); return true;
    default: return false;
  }
}

template <class P>
cudaError_t launch_mix_p(const efft_plan_s* p, const Pass& ps, void* data, const Batch& bt, cudaStream_t st) {
  MixArgs m;
  std::memset(&m, 0, sizeof(m));
  m.N = p->n;
  m.s = ps.s_int;
  m.L = ps.L_int;
  m.R = (int)ps.R_int;
  m.C = ps.C_int;
  m.log2C = __builtin_ctz((unsigned)ps.C_int);
  m.nrad = ps.nrad;
  for (int i = 0; i < ps.nrad; ++i) m.rad[i] = ps.rad[i];
  m.twB = p->twB;
  m.tw_lo = p->tw_lo;
  m.tw_hi = p->tw_hi;
  m.state = bt.state;
  m.ptrs = bt.ptrs;
  const uint32_t conj = (p->sign > 0) ? 1u : 0u;
  m.conj_in = (ps.kind == FIRST || ps.kind == SINGLE) ? conj : 0u;
  m.conj_out = (ps.kind == LAST || ps.kind == SINGLE) ? conj : 0u;
  // 1/N = 1/(M 2^e): the power of two here, 1/M is not exact and is not offered
  m.out_shift = ((p->flags & EFFT_FLAG_NORMALIZE) && (ps.kind == LAST || ps.kind == SINGLE)) ? p->log2n : 0;
  // middle pass, R = M * 2^b with b >= 4, power-of-two stride, C <= 32
  const uint64_t odd = ps.R_int / (ps.R_int & (~ps.R_int + 1));
  m.log2b = __builtin_ctzll(ps.R_int);
  m.log2s = __builtin_ctzll(ps.s_int);
  if (ps.kind == MID && odd == 3 && m.log2b >= 4 && m.log2b <= 6 && m.log2s >= 4 &&
      (ps.s_int & (ps.s_int - 1)) == 0 &&
      launch_m3_b<P>(m.log2b, m, p, data, bt.count, st))
    return cudaGetLastError();
  if (ps.kind == MID && odd > 1 && m.log2b >= 4 && (ps.s_int & (ps.s_int - 1)) == 0 && ps.C_int <= 32 &&
      launch_mixm_odd<P>((int)odd, m, ps, data, bt.count, st))
    return cudaGetLastError();
  switch (ps.kind) {
    case FIRST: launch_mix_kind<P, FIRST>(m, ps, data, bt.count, st); break;
    case MID: launch_mix_kind<P, MID>(m, ps, data, bt.count, st); break;
    case LAST: launch_mix_kind<P, LAST>(m, ps, data, bt.count, st); break;
    default: launch_mix_kind<P, SINGLE>(m, ps, data, bt.count, st); break;
  }
  return cudaGetLastError();
}


}  // namespace

namespace efft {
namespace host {

cudaError_t mix_set_attrs() {
  // two padded buffers of the tile plus R <= tile roots (float4)
  const int mix128 = 2 * (kMixTileC128 + kMixTileC128 / 16) * (int)sizeof(cdf2) + kMixTileC128 * (int)sizeof(float4);
  const int mix64 = 2 * (kMixTileC64 + kMixTileC64 / 16) * (int)sizeof(float2) + kMixTileC64 * (int)sizeof(float4);
  const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e[8] = {cudaFuncSetAttribute(efft_pass_mix<PolicyDF2, FIRST>, attr, mix128),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyDF2, MID>, attr, mix128),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyDF2, LAST>, attr, mix128),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyDF2, SINGLE>, attr, mix128),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyF32, FIRST>, attr, mix64),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyF32, MID>, attr, mix64),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyF32, LAST>, attr, mix64),
                      cudaFuncSetAttribute(efft_pass_mix<PolicyF32, SINGLE>, attr, mix64)};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  const cudaError_t f[14] = {
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 3>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 5>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 7>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 9>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 11>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 13>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyDF2, 15>, attr, mix128),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 3>, attr, mix64),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 5>, attr, mix64),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 7>, attr, mix64),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 9>, attr, mix64),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 11>, attr, mix64),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 13>, attr, mix64),
      cudaFuncSetAttribute(efft_pass_mixm<PolicyF32, 15>, attr, mix64)};
  for (cudaError_t x : f)
    if (x != cudaSuccess) return x;
  const cudaError_t g[6] = {
      cudaFuncSetAttribute(efft_pass_m3<PolicyDF2, 3>, attr, m3_smem_bytes(48, PolicyDF2::kElemBytes)),
      cudaFuncSetAttribute(efft_pass_m3<PolicyDF2, 6>, attr, m3_smem_bytes(96, PolicyDF2::kElemBytes)),
      cudaFuncSetAttribute(efft_pass_m3<PolicyDF2, 12>, attr, m3_smem_bytes(192, PolicyDF2::kElemBytes)),
      cudaFuncSetAttribute(efft_pass_m3<PolicyF32, 3>, attr, m3_smem_bytes(48, PolicyF32::kElemBytes)),
      cudaFuncSetAttribute(efft_pass_m3<PolicyF32, 6>, attr, m3_smem_bytes(96, PolicyF32::kElemBytes)),
      cudaFuncSetAttribute(efft_pass_m3<PolicyF32, 12>, attr, m3_smem_bytes(192, PolicyF32::kElemBytes))};
  for (cudaError_t x : g)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

cudaError_t launch_mix(const efft_plan_s* p, const Pass& ps, void* data, const Batch& bt, cudaStream_t st) {
  return (p->dtype == EFFT_C128) ? launch_mix_p<PolicyDF2>(p, ps, data, bt, st)
                                 : launch_mix_p<PolicyF32>(p, ps, data, bt, st);
}

}  // namespace host
}  // namespace efft
