// kernels.h -- host-side launch interface between the library's translation
// units (stencil kernels, Krylov kernels, the C ABI driver). Internal; not
// part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "jfnk.h"

#include "pdes.cuh"

namespace jfnk {

enum VType { VT_F64 = 0, VT_F32 = 1, VT_BF16 = 2 };
inline size_t vt_size(int t) { return t == VT_F64 ? 8 : (t == VT_F32 ? 4 : 2); }
// Fields per cell of a PDE (jfnk_pde).
inline int pde_nfields(int pde) {
  if (pde == JFNK_MAXWELL_VEC2D) return 4;
  return (pde == JFNK_SU_OLSON2D || pde == JFNK_MAXWELL_TE2D || pde == JFNK_BURGERS2D) ? 2 : 1;
}
// Planes of the source array aux[1] of a problem (Maxwell: Re, Im of f; the
// vector form: Re J_x, Im J_x, Re J_y, Im J_y).
inline int pde_source_planes(int pde) {
  return pde == JFNK_MAXWELL_VEC2D ? 4 : (pde == JFNK_MAXWELL_TE2D ? 2 : 0);
}

// Device workspace of one reduction site (partials + arrival counter).
struct RedWs {
  void* partials;          // kMaxVecBlocks-or-more blocks x kMaxK accumulators (8 bytes each)
  unsigned int* counter;   // zero between launches
  int max_blocks;          // capacity of partials in blocks
};

// Scalar post-processing done by the last block of a reduction (thread 0).
enum PostOp {
  POST_NONE = 0,
  POST_GMRES_RESTART = 1,   // sums[0] = ||r||^2: set beta, scale[0], g[0], convergence
  POST_NORM_EPS = 2,        // sums -> FD step into post_arg (see krylov.cu)
};

// Stencil geometry shared by all stencil kernels of a problem.
struct StencilGeom {
  dim3 block, grid;
  int rows_per_thread;     // R: each thread handles R rows strided by blockDim.y
  int nblocks;             // grid.x * grid.y
  int max_blocks;          // largest grid of any stencil launch form of the problem (reduction capacity)
};
StencilGeom stencil_geom(const ProbDev& P);

// Validate a problem and derive the kernels' constants (aux pointers left
// null); on failure *why (may be null) says what is wrong.
bool make_probdev(const jfnk_problem* pr, ProbDev* P, std::string* why);

struct LsCtl;
// F = F(x + alpha d; b) in precision t (x, d, b, F, xout of type t; d, b,
// F, xout, x32 may be null). sums[0] = ||F||^2, sums[1] = ||x + alpha d||^2
// (double) when sums != null. With ls (and sums) not null the launch is a
// line-search trial: alpha is ls->alpha, the kernel does nothing once
// ls->done is set, and its last block applies the Armijo decision (LsCtl).
cudaError_t launch_residual(const ProbDev& P, int t, const void* x, const void* d, double alpha,
                            const void* b, void* F, void* xout, float* x32, RedWs red, double* sums,
                            cudaStream_t st, LsCtl* ls = nullptr);

// The problem's right preconditioner at the state x (precision t): out =
// M^-1(x) v node by node (out may equal v, or be null) and, when sums is set,
// sums[0] = ||M^-1(x) v||^2. cudaErrorInvalidValue for a PDE without one.
cudaError_t launch_precond(const ProbDev& P, int t, const void* x, const void* v, void* out, double* sums, double beta,
                           RedWs red, cudaStream_t st);

// b = M(xn) + (1 - theta) dt G(xn) in precision t.
cudaError_t launch_rhs(const ProbDev& P, int t, const void* xn, void* b, cudaStream_t st);

// Jacobian-vector product in precision t (x, b, F, out, add, dw of type t;
// v of type tv = t or BF16 when t = FP32).
//   AD: (F, Jv) by one dual-number sweep; FD: Jv = (F(x + eps s v) - Fx)/eps.
//   The direction is s v with s = *vscale (null: 1).
//   out = c_jv * Jv + c_add * add (add may be null); F (AD only) may be null.
//   ndots in 0..3 reductions of out . dw[k] (dw[k] null: out . out) into
//   sums[k] (double), then the post-operation `post` on the last block.
// FD step: eps_fixed > 0 uses it; else rule 0 (scaled):
//   eps = sqrt(eps_mach)(1 + sqrt(*xn2)) / (sqrt(*vn2) s), vn2 null meaning
//   ||v|| = 1 after scaling; rule 1 (paper): sqrt(eps_mach) max(1, sqrt(*xn2)).
struct JvpArgs {
  int lin;                     // 0 AD, 1 FD
  int t, tv;
  const void* x; const void* v; const double* vscale;
  const void* b; void* F; const void* Fx;
  void* out; double c_jv; const void* add; double c_add;
  int ndots; const void* dw[3]; double* sums;
  int post; void* post_arg;
  double eps_fixed; int eps_rule; const double* xn2; const double* vn2;
  float* eps_out;              // FD: the step used (for reporting), may be null
  const int* active;           // device flag: the kernel does nothing when *active == 0 (null: always run)
  unsigned int* err;           // device error word for bounded waits of the staged sweep (null: not staged)
  int pdl;                     // staged sweep: programmatic launch after the previous kernel in the stream,
                               // which must not write x (the sweep loads x before its dependency wait)
  int precond;                 // the direction is M^-1 v (the problem's right preconditioner, gather form)
  double pbeta;                // its damping
};
cudaError_t launch_jvp(const ProbDev& P, const JvpArgs& a, RedWs red, cudaStream_t st);

// Adaptive time step of the 2D Burgers problem from the state x (precision
// t, fields u and v): *dt_out = C min(hx / max|u|, hy / max|v|,
// 1 / (2 nu (1/hx^2 + 1/hy^2))), terms with a zero denominator left out
// (none left: +Inf); NaN when x holds a non-finite value. Grid: at most
// 4 nsm blocks of 256 threads, partials in red.
cudaError_t launch_cfl_dt(const ProbDev& P, int t, const void* x, double* dt_out, RedWs red, int nsm,
                          cudaStream_t st);

}  // namespace jfnk
