// k_mixed_64.cu -- the MIXED-form window kernel's instantiations for 64-thread windows.
#include "k_mixed_nt.cuh"

namespace dich {

cudaError_t launch_window_mixed_64(int grid, size_t smem, cudaStream_t st, const WinArgs& a, int grid_y) {
  return launch_kind<64>(grid, grid_y, smem, st, a);
}

}  // namespace dich
