// stencil_allen_cahn.cu -- the stencil sweeps of AllenCahn2D (all launch forms,
// precisions and modes), in a translation unit of their own.
#include "stencil_impl.cuh"

namespace jfnk {

cudaError_t stencil_allen_cahn(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                         cudaStream_t st) {
  return stencil_dispatch<AllenCahn2D>(mode, P, t, tv, a, red, st);
}

}  // namespace jfnk
