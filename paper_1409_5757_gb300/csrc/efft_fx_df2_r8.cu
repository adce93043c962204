// efft_fx_df2_r8.cu -- the complex128 pass kernels with radix-8 register
// stages (8 values per thread, twice the threads of the radix-16 kernels on
// the same tile, so twice the resident warps: 32 per SM).  A translation unit
// of its own so that the kernel variants compile in parallel.
#include <cuda_runtime.h>

#include "efft_kernels.cuh"

namespace efft {
namespace {

constexpr int kLog2Cta = 12;  // 4096-element tiles, 512 threads, two CTAs per SM

template <int KIND, int LR>
constexpr auto tile_kernel() {
  return efft_pass_fx<PolicyDF2, KIND, LR, kLog2Cta - LR, 2, 0, 3>;
}
// 8192-element tiles, 1024 threads, one CTA per SM: the wide first pass and
// the strided last pass
template <int KIND, int LR>
constexpr auto wide_kernel() {
  return efft_pass_fx<PolicyDF2, KIND, LR, kLog2CtaWide - LR, 1, 0, 3>;
}
// swapping middle passes (clusters of two CTAs)
template <int LR, int SWLT, int MINB>
constexpr auto swap_kernel() {
  return efft_pass_fx<PolicyDF2, MID, LR, 2 * SWLT, MINB, SWLT, 3>;
}

template <class K>
void set_smem(K k, int elems, cudaError_t& err) {
  const cudaError_t x = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((elems + elems / 16 + 1) * PolicyDF2::kElemBytes));
  if (x != cudaSuccess && err == cudaSuccess) err = x;
}

template <class K>
cudaError_t launch(K k, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data, const PassArgs& a,
                   bool cluster) {
  if (!cluster) {
    k<<<grid, block, smem, st>>>(data, a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, data, a);
}

template <int KIND>
void tile_attrs(cudaError_t& err) {
  set_smem(tile_kernel<KIND, 8>(), 4096, err);
  set_smem(tile_kernel<KIND, 9>(), 4096, err);
  set_smem(tile_kernel<KIND, 10>(), 4096, err);
  set_smem(tile_kernel<KIND, 11>(), 4096, err);
}

template <int KIND>
cudaError_t tile_launch(int log2R, dim3 g, dim3 b, size_t sm, cudaStream_t st, void* d, const PassArgs& a) {
  switch (log2R) {
    case 8: return launch(tile_kernel<KIND, 8>(), g, b, sm, st, d, a, false);
    case 9: return launch(tile_kernel<KIND, 9>(), g, b, sm, st, d, a, false);
    case 10: return launch(tile_kernel<KIND, 10>(), g, b, sm, st, d, a, false);
    case 11: return launch(tile_kernel<KIND, 11>(), g, b, sm, st, d, a, false);
    default: return cudaErrorInvalidConfiguration;
  }
}

}  // namespace

cudaError_t fx_set_attrs_df2_r8() {
  cudaError_t err = cudaSuccess;
  tile_attrs<FIRST>(err);
  tile_attrs<MID>(err);
  tile_attrs<LAST>(err);
  set_smem(wide_kernel<FIRST, 10>(), 8192, err);
  set_smem(wide_kernel<FIRST, 11>(), 8192, err);
  set_smem(wide_kernel<LASTS, 9>(), 8192, err);
  set_smem(wide_kernel<LASTS, 10>(), 8192, err);
  set_smem(wide_kernel<LASTS, 11>(), 8192, err);
  set_smem(swap_kernel<11, 1, 1>(), 8192, err);
  set_smem(swap_kernel<10, 1, 2>(), 4096, err);
  set_smem(swap_kernel<8, 2, 2>(), 4096, err);
  return err;
}

bool fx_launch_df2_r8(int kind, int log2R, int log2C, int swap, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      void* data, const PassArgs& a) {
  cudaError_t e = cudaErrorInvalidConfiguration;
  const bool wide = (log2R + log2C == kLog2CtaWide);
  if (swap) {
    if (log2R == 11 && log2C == 2) e = launch(swap_kernel<11, 1, 1>(), grid, block, smem, st, data, a, true);
    else if (log2R == 10 && log2C == 2) e = launch(swap_kernel<10, 1, 2>(), grid, block, smem, st, data, a, true);
    else if (log2R == 8 && log2C == 4) e = launch(swap_kernel<8, 2, 2>(), grid, block, smem, st, data, a, true);
  } else if (wide && kind == FIRST) {
    if (log2R == 10) e = launch(wide_kernel<FIRST, 10>(), grid, block, smem, st, data, a, false);
    else if (log2R == 11) e = launch(wide_kernel<FIRST, 11>(), grid, block, smem, st, data, a, false);
  } else if (wide && kind == LASTS) {
    if (log2R == 9) e = launch(wide_kernel<LASTS, 9>(), grid, block, smem, st, data, a, false);
    else if (log2R == 10) e = launch(wide_kernel<LASTS, 10>(), grid, block, smem, st, data, a, false);
    else if (log2R == 11) e = launch(wide_kernel<LASTS, 11>(), grid, block, smem, st, data, a, false);
  } else if (log2R + log2C == kLog2Cta) {
    if (kind == FIRST) e = tile_launch<FIRST>(log2R, grid, block, smem, st, data, a);
    else if (kind == MID) e = tile_launch<MID>(log2R, grid, block, smem, st, data, a);
    else if (kind == LAST) e = tile_launch<LAST>(log2R, grid, block, smem, st, data, a);
  }
  return e == cudaSuccess;
}

}  // namespace efft
