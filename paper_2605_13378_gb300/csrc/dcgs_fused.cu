// dcgs_fused.cu -- host side of the fused delayed-CGS2 pass (dcgs_fused.cuh)
// for the 2D PDEs whose cells use face neighbours only: Allen-Cahn, the
// Maxwell TE problem and 2D Burgers.
#include "dcgs_fused.cuh"
#include "krylov.h"

namespace jfnk {

static bool fused_pde(int pde) { return pde == JFNK_ALLEN_CAHN2D || pde == JFNK_MAXWELL_TE2D || pde == JFNK_BURGERS2D; }

bool dcgs_fused_supported(const ProbDev& P, int m, int nsm) {
  if (!fused_pde(P.pde) || m < 1 || m > kMaxM) return false;
  FusedGeom g;
  // the widest stages of a cycle: step m - 2 with the JVP, step m - 1 without
  if (m >= 2 && !fused_geom(P.nx, P.ny, P.nf, m - 2, true, nsm, &g)) return false;
  return fused_geom(P.nx, P.ny, P.nf, m - 1, false, nsm, &g);
}

cudaError_t launch_dcgs_fused(const ProbDev& P, long long n, void* V, int j, bool has_w, bool wmul_one,
                              const void* U_in, void* U_out, const void* W_in, void* W_out, const void* X,
                              GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st) {
  FusedArgs a;
  if (!fused_pde(P.pde) || j < 0 || j >= kMaxM || n != P.ncell * P.nf) return cudaErrorInvalidValue;
  if (!fused_geom(P.nx, P.ny, P.nf, j, has_w, nsm, &a.g)) return cudaErrorInvalidValue;
  if (a.g.grid > red.max_blocks) return cudaErrorInvalidValue;
  a.n = n;
  a.ncell = P.ncell;
  a.nx = P.nx;
  a.ny = P.ny;
  a.j = j;
  a.has_w = has_w ? 1 : 0;
  a.wmul_one = wmul_one ? 1 : 0;
  a.V = (float*)V;
  a.U_in = (const float*)U_in;
  a.U_out = (float*)U_out;
  a.W_in = (const float*)W_in;
  a.W_out = (float*)W_out;
  a.X = (const float*)X;
  a.ctl = ctl;
  a.partials = (double*)red.partials;
  a.counter = red.counter;
  a.cap = red.max_blocks;
  a.err = err;
  switch (P.pde) {
    case JFNK_ALLEN_CAHN2D: return dcgs_fused_allen_cahn(a, P, st);
    case JFNK_MAXWELL_TE2D: return dcgs_fused_maxwell(a, P, st);
    case JFNK_BURGERS2D: return dcgs_fused_burgers2d(a, P, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace jfnk
