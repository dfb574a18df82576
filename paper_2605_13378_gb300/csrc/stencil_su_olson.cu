// stencil_su_olson.cu -- the stencil sweeps of SuOlson2D (all launch forms,
// precisions and modes), in a translation unit of their own.
#include "stencil_impl.cuh"

namespace jfnk {

cudaError_t stencil_su_olson(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                         cudaStream_t st) {
  return stencil_dispatch<SuOlson2D>(mode, P, t, tv, a, red, st);
}

}  // namespace jfnk
