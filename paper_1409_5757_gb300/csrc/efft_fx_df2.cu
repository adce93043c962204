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

// Swapping middle passes (clusters of two CTAs): R = 2^11 and 2^10 on 2 x 2
// column tiles (8192 and 4096 elements), R = 2^8 on 4 x 4 (4096 elements).
template <int LR, int SWLT, int MINB>
constexpr auto swap_kernel() {
  return efft_pass_fx<PolicyDF2, MID, LR, 2 * SWLT, MINB, SWLT>;
}
// Strided last passes on 8192-element tiles, one CTA per SM.
template <int LR>
constexpr auto lasts_kernel() {
  return efft_pass_fx<PolicyDF2, LASTS, LR, kLog2CtaWide - LR, 1>;
}

template <class K>
void set_smem(K k, int elems, cudaError_t& err) {
  const cudaError_t x = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((elems + elems / 16 + 1) * PolicyDF2::kElemBytes));
  if (x != cudaSuccess && err == cudaSuccess) err = x;
}

template <class K>
cudaError_t launch_cluster2(K k, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data, const PassArgs& a) {
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

// Persistent prefetching passes: 8192-element tiles (one CTA per SM) for
// the wide first pass, the strided last pass and the 2^11 swapping middle
// pass; 4096-element tiles (two CTAs per SM) for the other middle passes.
template <int KIND, int LR, int LC, int MINB, int SWLT = 0>
constexpr auto pf_kernel() {
  return efft_pass_pf<KIND, LR, LC, MINB, SWLT>;
}

template <class K>
cudaError_t launch_plain(K k, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data, const PassArgs& a) {
  k<<<grid, block, smem, st>>>(data, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t fx_set_attrs_df2_pf() {
  cudaError_t err = cudaSuccess;
  set_smem(pf_kernel<FIRST, 10, 3, 1>(), 8192, err);
  set_smem(pf_kernel<FIRST, 11, 2, 1>(), 8192, err);
  set_smem(pf_kernel<MID, 8, 4, 2>(), 4096, err);
  set_smem(pf_kernel<MID, 9, 3, 2>(), 4096, err);
  set_smem(pf_kernel<MID, 10, 2, 2>(), 4096, err);
  set_smem(pf_kernel<MID, 11, 1, 2>(), 4096, err);
  set_smem(pf_kernel<MID, 11, 2, 1, 1>(), 8192, err);
  set_smem(pf_kernel<MID, 10, 2, 2, 1>(), 4096, err);
  set_smem(pf_kernel<MID, 8, 4, 2, 2>(), 4096, err);
  set_smem(pf_kernel<LASTS, 9, 4, 1>(), 8192, err);
  set_smem(pf_kernel<LASTS, 10, 3, 1>(), 8192, err);
  set_smem(pf_kernel<LASTS, 11, 2, 1>(), 8192, err);
  return err;
}

bool fx_launch_df2_pf(int kind, int log2R, int log2C, int swap, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      void* data, const PassArgs& a) {
  cudaError_t e = cudaErrorInvalidConfiguration;
  if (swap) {
    if (log2R == 11 && log2C == 2) e = launch_cluster2(pf_kernel<MID, 11, 2, 1, 1>(), grid, block, smem, st, data, a);
    else if (log2R == 10 && log2C == 2) e = launch_cluster2(pf_kernel<MID, 10, 2, 2, 1>(), grid, block, smem, st, data, a);
    else if (log2R == 8 && log2C == 4) e = launch_cluster2(pf_kernel<MID, 8, 4, 2, 2>(), grid, block, smem, st, data, a);
  } else if (kind == FIRST) {
    if (log2R == 10 && log2C == 3) e = launch_plain(pf_kernel<FIRST, 10, 3, 1>(), grid, block, smem, st, data, a);
    else if (log2R == 11 && log2C == 2) e = launch_plain(pf_kernel<FIRST, 11, 2, 1>(), grid, block, smem, st, data, a);
  } else if (kind == MID) {
    if (log2R == 8 && log2C == 4) e = launch_plain(pf_kernel<MID, 8, 4, 2>(), grid, block, smem, st, data, a);
    else if (log2R == 9 && log2C == 3) e = launch_plain(pf_kernel<MID, 9, 3, 2>(), grid, block, smem, st, data, a);
    else if (log2R == 10 && log2C == 2) e = launch_plain(pf_kernel<MID, 10, 2, 2>(), grid, block, smem, st, data, a);
    else if (log2R == 11 && log2C == 1) e = launch_plain(pf_kernel<MID, 11, 1, 2>(), grid, block, smem, st, data, a);
  } else if (kind == LASTS) {
    if (log2R == 9 && log2C == 4) e = launch_plain(pf_kernel<LASTS, 9, 4, 1>(), grid, block, smem, st, data, a);
    else if (log2R == 10 && log2C == 3) e = launch_plain(pf_kernel<LASTS, 10, 3, 1>(), grid, block, smem, st, data, a);
    else if (log2R == 11 && log2C == 2) e = launch_plain(pf_kernel<LASTS, 11, 2, 1>(), grid, block, smem, st, data, a);
  }
  return e == cudaSuccess;
}

cudaError_t fx_set_attrs_df2() {
  cudaError_t err = cudaSuccess;
  attrs<FIRST>(err);
  attrs<MID>(err);
  attrs<LAST>(err);
  attrs_wide(err);
  set_smem(swap_kernel<11, 1, 1>(), 8192, err);
  set_smem(swap_kernel<10, 1, 2>(), 4096, err);
  set_smem(swap_kernel<8, 2, 2>(), 4096, err);
  set_smem(lasts_kernel<9>(), 8192, err);
  set_smem(lasts_kernel<10>(), 8192, err);
  set_smem(lasts_kernel<11>(), 8192, err);
  const cudaError_t e2 = fx_set_attrs_df2_pf();
  if (e2 != cudaSuccess && err == cudaSuccess) err = e2;
  return err;
}

bool fx_launch_df2_swap(int log2R, int log2C, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                        const PassArgs& a) {
  cudaError_t e;
  if (log2R == 11 && log2C == 2) e = launch_cluster2(swap_kernel<11, 1, 1>(), grid, block, smem, st, data, a);
  else if (log2R == 10 && log2C == 2) e = launch_cluster2(swap_kernel<10, 1, 2>(), grid, block, smem, st, data, a);
  else if (log2R == 8 && log2C == 4) e = launch_cluster2(swap_kernel<8, 2, 2>(), grid, block, smem, st, data, a);
  else return false;
  return e == cudaSuccess;
}

bool fx_launch_df2_lasts(int log2R, dim3 grid, dim3 block, size_t smem, cudaStream_t st, void* data,
                         const PassArgs& a) {
  switch (log2R) {
    case 9: lasts_kernel<9>()<<<grid, block, smem, st>>>(data, a); return true;
    case 10: lasts_kernel<10>()<<<grid, block, smem, st>>>(data, a); return true;
    case 11: lasts_kernel<11>()<<<grid, block, smem, st>>>(data, a); return true;
    default: return false;
  }
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
