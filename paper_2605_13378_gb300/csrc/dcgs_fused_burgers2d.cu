// dcgs_fused_burgers2d.cu -- the fused delayed-CGS2 pass of Burgers2D (one translation unit per PDE).
#include "dcgs_fused.cuh"

namespace jfnk {
cudaError_t dcgs_fused_burgers2d(const FusedArgs& a, const ProbDev& P, cudaStream_t st) {
  return dcgs_fused_dispatch<Burgers2D>(a, P, st);
}
}  // namespace jfnk
