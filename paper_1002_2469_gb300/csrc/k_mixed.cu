// k_mixed.cu -- instantiations of the MIXED-form window kernel (two blocks per thread, packed FP32x2).
#include "launch.cuh"

namespace dich {

// ADJ: the adjoint's instantiation (gradient sums in the store loop), chosen by a.xf
template <int NT, bool ADJ>
static cudaError_t launch_one(int grid, int grid_y, size_t smem, cudaStream_t st, const WinArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_window2<NT, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  return cudaLaunchKernelEx(&cfg, k_window2<NT, ADJ>, a);
}

cudaError_t launch_window_mixed(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y) {
  const bool adj = (a.xf != nullptr);
  switch (NT) {
    case 64: return adj ? launch_one<64, true>(grid, grid_y, smem, st, a) : launch_one<64, false>(grid, grid_y, smem, st, a);
    case 128: return adj ? launch_one<128, true>(grid, grid_y, smem, st, a) : launch_one<128, false>(grid, grid_y, smem, st, a);
    case 256: return adj ? launch_one<256, true>(grid, grid_y, smem, st, a) : launch_one<256, false>(grid, grid_y, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dich
