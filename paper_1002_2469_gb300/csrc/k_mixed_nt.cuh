// k_mixed_nt.cuh -- launch helpers of the MIXED-form window kernel (two blocks per thread, packed
// FP32x2), included by the translation units that instantiate it for one CTA width each
// (k_mixed_64.cu, k_mixed_128.cu, k_mixed_256.cu: compiled in parallel).
#pragma once
#include "launch.cuh"

namespace dich {

// KIND: the adjoint's instantiations (gradient sums in the store loop) when a.xf is set, else the
// forward ones; the register-path kind when a.bulk allows bulk copies, else the shared-memory one
// (six CTAs per SM)
template <int NT, int KIND>
static cudaError_t launch_one(int grid, int grid_y, size_t smem, cudaStream_t st, const WinArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_window2<NT, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, grid_y);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_window2<NT, KIND>, a);
}

template <int NT>
static cudaError_t launch_kind(int grid, int grid_y, size_t smem, cudaStream_t st, const WinArgs& a) {
  if (a.xf != nullptr)
    return a.bulk ? launch_one<NT, KIND_REGADJ>(grid, grid_y, smem, st, a) : launch_one<NT, KIND_ADJ>(grid, grid_y, smem, st, a);
  if (a.bulk) return launch_one<NT, KIND_REG>(grid, grid_y, smem, st, a);
  return launch_one<NT, KIND_SMEM>(grid, grid_y, smem, st, a);
}

}  // namespace dich
