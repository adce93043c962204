// efft_fx_f32.cu -- instantiations and launches of the specialised pass kernel for
// complex64 (FP32, 8192 elements per CTA).  A translation unit of its own so that the kernel variants compile
// in parallel.
#include <cuda_runtime.h>

#include "efft_fx32.cuh"
#include "efft_host.h"
#include "efft_kernels.cuh"

namespace efft {
namespace {

constexpr int kLog2Cta = 13;

template <int KIND>
void attrs(cudaError_t& err) {
  const int bytes = (int)(((1 << kLog2Cta) + (1 << kLog2Cta) / 16 + 1) * PolicyF32::kElemBytes);
  cudaError_t e[4] = {
      cudaFuncSetAttribute(efft_pass_fx<PolicyF32, KIND, 8, kLog2Cta - 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyF32, KIND, 9, kLog2Cta - 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyF32, KIND, 10, kLog2Cta - 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyF32, KIND, 11, kLog2Cta - 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)};
  for (cudaError_t x : e)
    if (x != cudaSuccess && err == cudaSuccess) err = x;
  const cudaError_t f = cudaFuncSetAttribute(efft_pass_fx32<KIND, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             fx32_smem_bytes(3));
  if (f != cudaSuccess && err == cudaSuccess) err = f;
}

template <int KIND>
bool launch(int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data, const PassArgs& a) {
  if (log2R == 10 && a.log2C == 3) {
    // 2^10 = 32 * 32: the radix-32 kernel, 256 threads on the same 8192-element tile
    efft_pass_fx32<KIND, 3><<<grid, 256, fx32_smem_bytes(3), st>>>(data, a);
    return true;
  }
  switch (log2R) {
    case 8: efft_pass_fx<PolicyF32, KIND, 8, kLog2Cta - 8><<<grid, block, smem, st>>>(data, a); return true;
    case 9: efft_pass_fx<PolicyF32, KIND, 9, kLog2Cta - 9><<<grid, block, smem, st>>>(data, a); return true;
    case 10: efft_pass_fx<PolicyF32, KIND, 10, kLog2Cta - 10><<<grid, block, smem, st>>>(data, a); return true;
    case 11: efft_pass_fx<PolicyF32, KIND, 11, kLog2Cta - 11><<<grid, block, smem, st>>>(data, a); return true;
    default: return false;
  }
}

}  // namespace

cudaError_t fx_set_attrs_f32() {
  cudaError_t err = cudaSuccess;
  attrs<FIRST>(err);
  attrs<MID>(err);
  attrs<LAST>(err);
  const cudaError_t w = cudaFuncSetAttribute(efft_pass_fx32<FIRST, kLog2CtaWideC64 - 10, 1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             fx32_smem_bytes(kLog2CtaWideC64 - 10));
  if (w != cudaSuccess && err == cudaSuccess) err = w;
  constexpr int elems = 1 << kLog2CtaWideC64;
  const cudaError_t m = cudaFuncSetAttribute(efft_pass_fx<PolicyF32, MID, 11, kLog2CtaWideC64 - 11, 1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (elems + elems / 16 + 1) * 8);
  if (m != cudaSuccess && err == cudaSuccess) err = m;
  const cudaError_t tm = cudaFuncSetAttribute(efft_pass_fx32_tma<kLog2CtaWideC64 - 10>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, fx32_tma_smem_bytes());
  if (tm != cudaSuccess && err == cudaSuccess) err = tm;
  const cudaError_t tm2 = cudaFuncSetAttribute(efft_pass_mid_tma_f32<11, kLog2CtaWideC64 - 11>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, mid_tma_smem_bytes());
  if (tm2 != cudaSuccess && err == cudaSuccess) err = tm2;
  return err;
}

bool fx_launch_f32_mid_tma(dim3 grid, cudaStream_t st, void* data, const PassArgs& a, const void* tensor_map) {
  constexpr int LC = kLog2CtaWideC64 - 11;
  const CUtensorMap& map = *static_cast<const CUtensorMap*>(tensor_map);
  efft_pass_mid_tma_f32<11, LC><<<grid, 1 << (11 + LC - 4), mid_tma_smem_bytes(), st>>>(data, a, map);
  return true;
}

bool fx_launch_f32_tma(dim3 grid, cudaStream_t st, void* data, const PassArgs& a, const void* tensor_map) {
  constexpr int LC = kLog2CtaWideC64 - 10;
  const CUtensorMap& map = *static_cast<const CUtensorMap*>(tensor_map);
  efft_pass_fx32_tma<LC><<<grid, 32 << LC, fx32_tma_smem_bytes(), st>>>(data, a, map);
  return true;
}

bool fx_launch_f32_wide(int kind, int log2R, dim3 grid, cudaStream_t st, void* data, const PassArgs& a) {
  if (kind == FIRST && log2R == 10 && a.log2C == kLog2CtaWideC64 - 10) {
    constexpr int LC = kLog2CtaWideC64 - 10;
    efft_pass_fx32<FIRST, LC, 1><<<grid, 32 << LC, fx32_smem_bytes(LC), st>>>(data, a);
    return true;
  }
  if (kind == MID && log2R == 11 && a.log2C == kLog2CtaWideC64 - 11) {
    constexpr int LC = kLog2CtaWideC64 - 11;
    constexpr int elems = 1 << kLog2CtaWideC64;
    efft_pass_fx<PolicyF32, MID, 11, LC, 1><<<grid, elems / 16, (elems + elems / 16 + 1) * 8, st>>>(data, a);
    return true;
  }
  return false;
}

bool fx_launch_f32(int kind, int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                   const PassArgs& a) {
  switch (kind) {
    case FIRST: return launch<FIRST>(log2R, grid, block, smem, st, data, a);
    case MID: return launch<MID>(log2R, grid, block, smem, st, data, a);
    case LAST: return launch<LAST>(log2R, grid, block, smem, st, data, a);
    default: return false;
  }
}

}  // namespace efft
