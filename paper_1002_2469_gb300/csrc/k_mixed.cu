// k_mixed.cu -- the MIXED-form window kernel's launch by CTA width (the instantiations live in
// k_mixed_64.cu, k_mixed_128.cu and k_mixed_256.cu).
#include "launch.cuh"

namespace dich {

cudaError_t launch_window_mixed_64(int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y);
cudaError_t launch_window_mixed_128(int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y);
cudaError_t launch_window_mixed_256(int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y);

cudaError_t launch_window_mixed(int NT, int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y) {
  switch (NT) {
    case 64: return launch_window_mixed_64(grid, smem, st, a, grid_y);
    case 128: return launch_window_mixed_128(grid, smem, st, a, grid_y);
    case 256: return launch_window_mixed_256(grid, smem, st, a, grid_y);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dich
