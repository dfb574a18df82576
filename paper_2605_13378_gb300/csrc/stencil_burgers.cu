// stencil_burgers.cu -- the stencil sweeps of Burgers1D (all launch forms,
// precisions and modes), in a translation unit of their own.
#include "stencil_impl.cuh"

namespace jfnk {

cudaError_t stencil_burgers(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                         cudaStream_t st) {
  return stencil_dispatch<Burgers1D>(mode, P, t, tv, a, red, st);
}

}  // namespace jfnk
