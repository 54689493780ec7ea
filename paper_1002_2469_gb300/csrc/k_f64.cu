// k_f64.cu -- FP64 instantiations of the window kernel.
#include "launch.cuh"

namespace dich {

template <int NT>
static cudaError_t launch_one(int grid, int grid_y, size_t smem, cudaStream_t st, const WinArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_window<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  return cudaLaunchKernelEx(&cfg, k_window<NT>, a);
}

cudaError_t launch_window_f64(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y) {
  switch (NT) {
    case 64: return launch_one<64>(grid, grid_y, smem, st, a);
    case 128: return launch_one<128>(grid, grid_y, smem, st, a);
    case 256: return launch_one<256>(grid, grid_y, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dich
