// batch_allen_cahn.cu -- batch kernels of the AllenCahn2D problem (one translation unit per PDE).
#include "batch_impl.cuh"

namespace jfnk {
cudaError_t batch_launch_allen_cahn(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  return batch_launch_pde<AllenCahn2D>(ts, tj, L, grid, st);
}
int batch_occ_allen_cahn(int ts, int tj) { return batch_occ_pde<AllenCahn2D>(ts, tj); }
}  // namespace jfnk
