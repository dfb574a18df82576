// stencil_maxwell_vec.cu -- the stencil sweeps of MaxwellVec2D (the paper's
// vector TE form; all precisions and modes, gather launch form), in a
// translation unit of their own.
#include "stencil_impl.cuh"

namespace jfnk {

cudaError_t stencil_maxwell_vec(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                                cudaStream_t st) {
  return stencil_dispatch<MaxwellVec2D>(mode, P, t, tv, a, red, st);
}

}  // namespace jfnk
