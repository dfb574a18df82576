// batch_su_olson.cu -- batch kernels of the SuOlson2D problem (one translation unit per PDE).
#include "batch_impl.cuh"

namespace jfnk {
cudaError_t batch_launch_su_olson(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  return batch_launch_pde<SuOlson2D>(ts, tj, L, grid, st);
}
int batch_occ_su_olson(int ts, int tj) { return batch_occ_pde<SuOlson2D>(ts, tj); }
}  // namespace jfnk
