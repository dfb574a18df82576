// batch_maxwell.cu -- batch kernels of the MaxwellTE2D problem (one translation unit per PDE).
#include "batch_impl.cuh"

namespace jfnk {
cudaError_t batch_launch_maxwell(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  return batch_launch_pde<MaxwellTE2D>(ts, tj, L, grid, st);
}
int batch_occ_maxwell(int ts, int tj) { return batch_occ_pde<MaxwellTE2D>(ts, tj); }
}  // namespace jfnk
