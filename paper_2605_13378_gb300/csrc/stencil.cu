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
    case 4: return stencil_burgers2d(mode, P, t, tv, a, red, st);
    case 5: return stencil_maxwell_vec(mode, P, t, tv, a, red, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_residual(const ProbDev& P, int t, const void* x, const void* d, double alpha, const void* b,
                            void* F, void* xout, float* x32, RedWs red, double* sums, cudaStream_t st, LsCtl* ls) {
  if (ls && !sums) return cudaErrorInvalidValue;   // the decision needs the reduced norm
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x; a.v = d; a.alpha = alpha; a.b = b; a.F = F; a.xout = xout; a.x32 = x32; a.sums = sums; a.ls = ls;
  return stencil_pde(SM_RESID, P, t, t, a, red, st);
}

cudaError_t launch_precond(const ProbDev& P, int t, const void* x, const void* v, void* out, double* sums, double beta,
                           RedWs red, cudaStream_t st) {
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x; a.v = v; a.out = out; a.sums = sums; a.pbeta = beta;
  return stencil_pde(SM_PREC, P, t, t, a, red, st);
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
  a.err = in.err;
  a.pdl = in.pdl;
  a.precond = in.precond;
  a.pbeta = in.pbeta;
  if (in.lin == 0) return stencil_pde(SM_AD, P, in.t, in.tv, a, red, st);
  return stencil_pde(SM_FD, P, in.t, in.tv, a, red, st);
}

// ---------------------------------------------------------------------------
// CFL step: per-block max|u|, max|v| (a non-finite value counts as +Inf),
// the last block combines the partials and evaluates the rule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cfl_abs(double a) {
  a = fabs(a);
  return a <= 1.7976931348623157e308 ? a : 1.0 / 0.0;
}

template <class T>
__global__ void __launch_bounds__(256) k_cfl_dt(const T* __restrict__ x, long long ncell, double hx, double hy,
                                                double nu, double C, double* partials, unsigned int* counter,
                                                double* dt_out) {
  double mu = 0.0, mv = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += stride) {
    mu = fmax(mu, cfl_abs((double)x[c]));
    mv = fmax(mv, cfl_abs((double)x[ncell + c]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
    mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
  }
  __shared__ double s_m[2][8];
  __shared__ unsigned int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_m[0][warp] = mu; s_m[1][warp] = mv; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a = fmax(a, s_m[0][w]); b = fmax(b, s_m[1][w]); }
    partials[(size_t)blockIdx.x * kMaxK + 0] = a;
    partials[(size_t)blockIdx.x * kMaxK + 1] = b;
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int k = lane; k < (int)gridDim.x; k += 32) {
    a = fmax(a, partials[(size_t)k * kMaxK + 0]);
    b = fmax(b, partials[(size_t)k * kMaxK + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if (lane == 0) {
    *dt_out = cfl_rule(a, b, hx, hy, nu, C);
    *counter = 0u;
  }
}

cudaError_t launch_cfl_dt(const ProbDev& P, int t, const void* x, double* dt_out, RedWs red, int nsm,
                          cudaStream_t st) {
  if (P.nf != 2 || (t != VT_F64 && t != VT_F32)) return cudaErrorInvalidValue;
  long long nb = (P.ncell + 1023) / 1024;
  const long long cap = 4LL * (nsm > 0 ? nsm : 1);
  if (nb > cap) nb = cap;
  if (nb > red.max_blocks) nb = red.max_blocks;
  if (nb < 1) return cudaErrorInvalidValue;
  double* part = (double*)red.partials;
  if (t == VT_F64)
    k_cfl_dt<double><<<(unsigned)nb, 256, 0, st>>>((const double*)x, P.ncell, P.hx, P.hy, P.p0, P.cfl, part,
                                                   red.counter, dt_out);
  else
    k_cfl_dt<float><<<(unsigned)nb, 256, 0, st>>>((const float*)x, P.ncell, P.hx, P.hy, P.p0, P.cfl, part,
                                                  red.counter, dt_out);
  return cudaGetLastError();
}

}  // namespace jfnk
