// dcgs_fused_allen_cahn.cu -- the fused delayed-CGS2 pass of AllenCahn2D (one translation unit per PDE).
#include "dcgs_fused.cuh"

namespace jfnk {
cudaError_t dcgs_fused_allen_cahn(const FusedArgs& a, const ProbDev& P, cudaStream_t st) {
  return dcgs_fused_dispatch<AllenCahn2D>(a, P, st);
}
}  // namespace jfnk
