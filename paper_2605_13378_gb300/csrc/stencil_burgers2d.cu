// stencil_burgers2d.cu -- the stencil sweeps of Burgers2D (all launch forms,
// precisions and modes), in a translation unit of their own.
#include "stencil_impl.cuh"

namespace jfnk {

cudaError_t stencil_burgers2d(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                           cudaStream_t st) {
  return stencil_dispatch<Burgers2D>(mode, P, t, tv, a, red, st);
}

}  // namespace jfnk
