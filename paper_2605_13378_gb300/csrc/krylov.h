// krylov.h -- host launch interface of the flat-vector Krylov kernels.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"
#include "ctl.cuh"

namespace jfnk {

// Vectors of one BiCGSTAB solve (JVP precision except F (state) and d).
struct BicgVecs {
  const void* F; void* r; void* rhat; void* p; void* v; void* s; void* t; void* d;
  const double* sums;   // init: sums[0] = ||F||^2
  double* pn2; double* sn2;
};

// One CGS2 pass (1: dots, 2: update + dots, 3: update + norm + Givens) of
// Arnoldi step k - 1 over basis vectors 0 .. k-1.
cudaError_t launch_arnoldi_pass(int pass, int tb, int tj, long long n, void* V, int k, void* w, GmresCtl* ctl,
                                RedWs red, cudaStream_t st);
cudaError_t launch_gmres_init(int ts, int tj, int tb, int td, long long n, const void* F, void* u0, void* rhs,
                              void* d, GmresCtl* ctl, const double* sums, double tol, int m, cudaStream_t st);
// back substitution + d += V y over at most kmax vectors
cudaError_t launch_gmres_finish(int tb, int td, long long n, const void* V, void* d, GmresCtl* ctl, int kmax,
                                cudaStream_t st, int streamed, unsigned int* err, int nsm);
// Streaming (bulk-copy) form of the basis passes: mode 1 dots, 2 update + dots,
// 3 update + norm + Givens (Arnoldi step k - 1), 4 solution update d += V y
// over ctl->k vectors (kmax an upper bound known to the host). nsm CTAs.
bool stream_supported(long long n);
cudaError_t basis_stream_f64(int mode, long long n, const void* V, int k, int kmax, void* w, void* d, GmresCtl* ctl,
                             RedWs red, unsigned int* err, int nsm, cudaStream_t st);
cudaError_t basis_stream_f32(int mode, int td, long long n, const void* V, int k, int kmax, void* w, void* d,
                             GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st);
cudaError_t basis_stream_bf16(int mode, long long n, const void* V, int k, int kmax, void* w, void* d,
                              GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st);
cudaError_t launch_basis_stream(int mode, int tb, int tj, int td, long long n, const void* V, int k, int kmax,
                                void* w, void* d, GmresCtl* ctl, RedWs red, unsigned int* err, int nsm,
                                cudaStream_t st);
// Delayed CGS2 (dcgs_impl.cuh, ctl.cuh dcgs_step): pass 1 the fused dots of
// Arnoldi step j over basis slots 0..j and w (w null: the last step of a
// cycle, which only completes column j - 1), pass 2 the fused update of step
// j. Requires stream_supported(n). defer: the coefficient step of step j runs at
// the start of its update pass, in every block, instead of at the end of its
// dots pass (w not null; the partials must hold 2 nsm blocks); both passes of
// the step take the same value.
cudaError_t dcgs_f64(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                     unsigned int* err, int nsm, cudaStream_t st, bool pdl = false, bool defer = false);
cudaError_t dcgs_f32(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                     unsigned int* err, int nsm, cudaStream_t st, bool pdl = false, bool defer = false);
cudaError_t dcgs_bf16(int pass, long long n, void* V, int j, const void* w, GmresCtl* ctl, RedWs red,
                      unsigned int* err, int nsm, cudaStream_t st, bool pdl = false, bool defer = false);
// Fused delayed-CGS2 Arnoldi pass for the AD JVP, FP32 basis and JVP, 2D
// PDEs with face neighbours only (Allen-Cahn, Maxwell TE, 2D Burgers):
// q_j -> basis slot j, u_{j+1} = U_out, J u_{j+1} -> W_out (when has_w), and
// the dots of step j + 1 with its Hessenberg step on the last CTA. u_j is read
// from U_in and w_j from W_in (times sigma_j unless wmul_one); X is the state
// in FP32. dcgs_fused_supported says whether every step of a GMRES(m) cycle
// fits the pass (nx % 4 == 0, ny >= 3, shared-memory plan).
bool dcgs_fused_supported(const ProbDev& P, int m, int nsm);
cudaError_t launch_dcgs_fused(const ProbDev& P, long long n, void* V, int j, bool has_w, bool wmul_one,
                              const void* U_in, void* U_out, const void* W_in, void* W_out, const void* X,
                              GmresCtl* ctl, RedWs red, unsigned int* err, int nsm, cudaStream_t st);

// pdl: launched programmatically after the kernel before it (see grid_dep_wait in stream.cuh)
cudaError_t launch_dcgs(int pass, int tb, int tj, long long n, void* V, int j, const void* w, GmresCtl* ctl,
                        RedWs red, unsigned int* err, int nsm, cudaStream_t st, bool pdl = false, bool defer = false);
cudaError_t launch_cast(int ti, int to, long long n, const void* x, void* y, double c, cudaStream_t st);
// Reset the line-search control of one Newton step (LsCtl): merit fnorm, trial alpha = 1.
cudaError_t launch_ls_begin(LsCtl* c, double fnorm, double c1, double min_alpha, int accept_first, cudaStream_t st);
cudaError_t launch_vdots(int t, long long n, int nd, const void* const* a, const void* const* b, double* sums,
                         RedWs red, const int* active, cudaStream_t st);
// CG: phase 0 init (r = p = -F, d = 0), 1 p = r + beta p (not in the first
// iteration), 2 after q = J p (vv.v) with p.q in c->sums[0]: x, r update,
// convergence, beta. vv.pn2 (may be null) gets ||p||^2 for the FD step.
cudaError_t launch_cg(int phase, int ts, int tj, int td, long long n, const BicgVecs& vv, BicgCtl* c, RedWs red,
                      int it, double tol, cudaStream_t st);
// phase 0 init, 1 p-update, 2 s-update, 3 half-step x update, 4 x/r update
cudaError_t launch_bicg(int phase, int ts, int tj, int td, long long n, const BicgVecs& vv, BicgCtl* c,
                        RedWs red, int it, double tol, cudaStream_t st);

}  // namespace jfnk
