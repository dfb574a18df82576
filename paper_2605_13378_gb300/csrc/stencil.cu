// stencil.cu -- launch geometry and the host entry points of the stencil
// sweeps (residual, right-hand side, AD and FD Jacobian-vector products).
// The kernels are in stencil_impl.cuh; each PDE is compiled in its own
// translation unit (stencil_<pde>.cu).
#include <string.h>

#include "stencil_impl.cuh"

namespace jfnk {

StencilGeom stencil_geom(const ProbDev& P) {
  StencilGeom g;
  if (P.ny == 1) {
    g.block = dim3(256, 1, 1);
  } else {
    g.block = dim3(32, 8, 1);
  }
  const long long gx = (P.nx + g.block.x - 1) / g.block.x;
  const long long rows = (P.ny + g.block.y - 1) / g.block.y;
  long long R = (gx * rows + 1215) / 1216;
  if (R < 1) R = 1;
  const long long gy = (rows + R - 1) / R;
  g.grid = dim3((unsigned)gx, (unsigned)gy, 1);
  g.rows_per_thread = (int)R;
  g.nblocks = (int)(gx * gy);
  // capacity needed by any launch form of this problem
  const int m4 = march_geom(P, 4).nblocks, m2 = march_geom(P, 2).nblocks;
  g.max_blocks = g.nblocks;
  if (m4 > g.max_blocks) g.max_blocks = m4;
  if (m2 > g.max_blocks) g.max_blocks = m2;
  return g;
}

static cudaError_t stencil_pde(int mode, const ProbDev& P, int t, int tv, const StencilArgs& a, RedWs red,
                               cudaStream_t st) {
  switch (P.pde) {
    case 0: return stencil_burgers(mode, P, t, tv, a, red, st);
    case 1: return stencil_allen_cahn(mode, P, t, tv, a, red, st);
    case 2: return stencil_su_olson(mode, P, t, tv, a, red, st);
    case 3: return stencil_maxwell(mode, P, t, tv, a, red, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_residual(const ProbDev& P, int t, const void* x, const void* d, double alpha, const void* b,
                            void* F, void* xout, float* x32, RedWs red, double* sums, cudaStream_t st) {
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x; a.v = d; a.alpha = alpha; a.b = b; a.F = F; a.xout = xout; a.x32 = x32; a.sums = sums;
  return stencil_pde(SM_RESID, P, t, t, a, red, st);
}

cudaError_t launch_rhs(const ProbDev& P, int t, const void* xn, void* b, cudaStream_t st) {
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.x = xn; a.out = b;
  return stencil_pde(SM_RHS, P, t, t, a, RedWs{nullptr, nullptr, 0}, st);
}

cudaError_t launch_jvp(const ProbDev& P, const JvpArgs& in, RedWs red, cudaStream_t st) {
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.x = in.x; a.v = in.v; a.vscale = in.vscale; a.b = in.b; a.F = in.F; a.Fx = in.Fx;
  a.out = in.out; a.c_jv = in.c_jv; a.add = in.add; a.c_add = in.c_add;
  a.ndots = in.ndots; a.dw[0] = in.dw[0]; a.dw[1] = in.dw[1]; a.dw[2] = in.dw[2]; a.sums = in.sums;
  a.post = in.post; a.post_arg = in.post_arg;
  a.eps_fixed = in.eps_fixed; a.eps_rule = in.eps_rule; a.xn2 = in.xn2; a.vn2 = in.vn2; a.eps_out = in.eps_out;
  a.active = in.active;
  if (in.lin == 0) return stencil_pde(SM_AD, P, in.t, in.tv, a, red, st);
  return stencil_pde(SM_FD, P, in.t, in.tv, a, red, st);
}

}  // namespace jfnk
