// batch_burgers2d.cu -- batch kernels of the Burgers2D problem (one translation unit per PDE).
#include "batch_impl.cuh"

namespace jfnk {
cudaError_t batch_launch_burgers2d(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  return batch_launch_pde<Burgers2D>(ts, tj, L, grid, st);
}
int batch_occ_burgers2d(int ts, int tj) { return batch_occ_pde<Burgers2D>(ts, tj); }
}  // namespace jfnk
