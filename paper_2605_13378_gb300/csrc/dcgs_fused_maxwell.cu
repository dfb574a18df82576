// dcgs_fused_maxwell.cu -- the fused delayed-CGS2 pass of MaxwellTE2D (one translation unit per PDE).
#include "dcgs_fused.cuh"

namespace jfnk {
cudaError_t dcgs_fused_maxwell(const FusedArgs& a, const ProbDev& P, cudaStream_t st) {
  return dcgs_fused_dispatch<MaxwellTE2D>(a, P, st);
}
}  // namespace jfnk
