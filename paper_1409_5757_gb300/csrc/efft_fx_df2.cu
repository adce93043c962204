// efft_fx_df2.cu -- instantiations and launches of the specialised pass kernel for
// complex128 (packed double-float, 4096 elements per CTA).  A translation unit of its own so that the kernel variants compile
// in parallel.
#include <cuda_runtime.h>

#include "efft_kernels.cuh"

namespace efft {
namespace {

constexpr int kLog2Cta = 12;

template <int KIND>
void attrs(cudaError_t& err) {
  const int bytes = (int)(((1 << kLog2Cta) + (1 << kLog2Cta) / 16 + 1) * PolicyDF2::kElemBytes);
  cudaError_t e[4] = {
      cudaFuncSetAttribute(efft_pass_fx<PolicyDF2, KIND, 8, kLog2Cta - 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyDF2, KIND, 9, kLog2Cta - 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyDF2, KIND, 10, kLog2Cta - 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyDF2, KIND, 11, kLog2Cta - 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)};
  for (cudaError_t x : e)
    if (x != cudaSuccess && err == cudaSuccess) err = x;
}

template <int KIND>
bool launch(int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data, const PassArgs& a) {
  switch (log2R) {
    case 8: efft_pass_fx<PolicyDF2, KIND, 8, kLog2Cta - 8><<<grid, block, smem, st>>>(data, a); return true;
    case 9: efft_pass_fx<PolicyDF2, KIND, 9, kLog2Cta - 9><<<grid, block, smem, st>>>(data, a); return true;
    case 10: efft_pass_fx<PolicyDF2, KIND, 10, kLog2Cta - 10><<<grid, block, smem, st>>>(data, a); return true;
    case 11: efft_pass_fx<PolicyDF2, KIND, 11, kLog2Cta - 11><<<grid, block, smem, st>>>(data, a); return true;
    default: return false;
  }
}

void attrs_wide(cudaError_t& err) {
  const int bytes = (int)(((1 << kLog2CtaWide) + (1 << kLog2CtaWide) / 16 + 1) * PolicyDF2::kElemBytes);
  cudaError_t e[2] = {
      cudaFuncSetAttribute(efft_pass_fx<PolicyDF2, FIRST, 10, kLog2CtaWide - 10, 1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
      cudaFuncSetAttribute(efft_pass_fx<PolicyDF2, FIRST, 11, kLog2CtaWide - 11, 1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)};
  for (cudaError_t x : e)
    if (x != cudaSuccess && err == cudaSuccess) err = x;
}

}  // namespace

cudaError_t fx_set_attrs_df2() {
  cudaError_t err = cudaSuccess;
  attrs<FIRST>(err);
  attrs<MID>(err);
  attrs<LAST>(err);
  attrs_wide(err);
  return err;
}

bool fx_launch_df2_wide(int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                        const PassArgs& a) {
  switch (log2R) {
    case 10:
      efft_pass_fx<PolicyDF2, FIRST, 10, kLog2CtaWide - 10, 1><<<grid, block, smem, st>>>(data, a);
      return true;
    case 11:
      efft_pass_fx<PolicyDF2, FIRST, 11, kLog2CtaWide - 11, 1><<<grid, block, smem, st>>>(data, a);
      return true;
    default: return false;
  }
}

bool fx_launch_df2(int kind, int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                   const PassArgs& a) {
  switch (kind) {
    case FIRST: return launch<FIRST>(log2R, grid, block, smem, st, data, a);
    case MID: return launch<MID>(log2R, grid, block, smem, st, data, a);
    case LAST: return launch<LAST>(log2R, grid, block, smem, st, data, a);
    default: return false;
  }
}

}  // namespace efft
