// Persistent whole-solve kernels, launch mode 2 (see gpe_persist.cuh).
#include "gpe_persist.cuh"
namespace gpe {
cudaError_t launch_persist_m2(int M, int dim, const PersistArgs& P, int grid, int block, size_t smem,
                              cudaStream_t st, int* max_blocks_per_sm) {
  return launch_persist_mode<2>(M, dim, P, grid, block, smem, st, max_blocks_per_sm);
}
}  // namespace gpe
