// batch_burgers.cu -- batch kernels of the Burgers1D problem (one translation unit per PDE).
#include "batch_impl.cuh"

namespace jfnk {
cudaError_t batch_launch_burgers(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  return batch_launch_pde<Burgers1D>(ts, tj, L, grid, st);
}
int batch_occ_burgers(int ts, int tj) { return batch_occ_pde<Burgers1D>(ts, tj); }
}  // namespace jfnk
