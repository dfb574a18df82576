// ctl.cuh -- device-resident control state of the Krylov solvers and the
// scalar steps that the last block of a reduction performs on it.
#pragma once

#include "common.cuh"

namespace jfnk {

constexpr int kMaxM = 64;   // largest GMRES restart length (JFNK_MAX_RESTART)

// Restarted GMRES(m) state of the current cycle. The basis is stored
// unnormalised: column t of V holds u_t, and v_t = scale[t] * u_t is the
// orthonormal Arnoldi vector, so no kernel ever rescales a basis vector.
struct GmresCtl {
  // scalar head (copied to the host after each cycle)
  double bnorm, target, beta, resid;
  int m;                           // restart length
  int k;                           // Arnoldi steps completed in this cycle
  int active;                      // 1 while the cycle iterates
  int converged, breakdown, nonfinite;
  int its;                         // Arnoldi steps over all cycles
  int pad_;
  volatile int* host_active;       // mapped host word mirroring `active` (may be null)
  // arrays
  double H[(kMaxM + 1) * kMaxM];   // Hessenberg, column-major H[j * (kMaxM + 1) + i], rotated in place
  double h1[kMaxM + 1];            // first Gram-Schmidt pass of column j
  double h2[kMaxM + 1];            // second pass
  double cs[kMaxM], sn[kMaxM];     // Givens rotations
  double g[kMaxM + 1];             // rotated right-hand side beta e_1
  double y[kMaxM];                 // least-squares solution at the end of a cycle
  double scale[kMaxM + 1];         // v_t = scale[t] u_t
};
constexpr size_t kGmresHeadBytes = 4 * sizeof(double) + 8 * sizeof(int) + sizeof(void*);

// BiCGSTAB / CG scalars (van der Vorst; Hestenes-Stiefel).
struct BicgCtl {
  double rho, rho_old, alpha, omega, beta;
  double bnorm, target, resid;
  double sums[4];                  // reduction results of the current phase
  int active, converged, breakdown, nonfinite, its;
  int flag_half;                   // it + 1 of an iteration that converged at its half step
  volatile int* host_active;       // mapped host word mirroring `active` (may be null)
};

__device__ __forceinline__ void mirror_active(volatile int* h, int a) {
  if (h) {
    *h = a;
    __threadfence_system();
  }
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// Start of a GMRES cycle from a residual r with ||r||^2 = r2: u_0 = r is
// already stored; set beta, scale[0], g[0] and the convergence test.
__device__ __forceinline__ void gmres_cycle_start(GmresCtl* c, double r2) {
  const double beta = sqrt(r2);
  c->k = 0;
  c->resid = beta;
  c->beta = beta;
  if (!finite_d(beta)) {
    c->nonfinite = 1;
    c->active = 0;
  } else if (beta <= c->target) {
    c->converged = 1;
    c->active = 0;
  } else {
    c->g[0] = beta;
    c->scale[0] = 1.0 / beta;
    c->active = 1;
  }
  mirror_active(c->host_active, c->active);
}

// Step j of Arnoldi after both Gram-Schmidt passes: column j of H is
// h1 + h2 with H[j+1, j] = ||u_{j+1}|| = sqrt(n2). Apply the previous
// rotations, form the new one, update g and test |g_{j+1}| <= tol ||b||.
__device__ __forceinline__ void gmres_givens_step(GmresCtl* c, int j, double n2) {
  double* col = c->H + (size_t)j * (kMaxM + 1);
  for (int i = 0; i <= j; ++i) col[i] = c->h1[i] + c->h2[i];
  const double hn = sqrt(n2);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = c->cs[i] * a + c->sn[i] * b;
    col[i + 1] = -c->sn[i] * a + c->cs[i] * b;
  }
  const double f = col[j], gg = col[j + 1];
  const double r = hypot(f, gg);
  double cs = 1.0, sn = 0.0;
  if (r != 0.0) { cs = f / r; sn = gg / r; }
  c->cs[j] = cs;
  c->sn[j] = sn;
  col[j] = cs * f + sn * gg;
  col[j + 1] = 0.0;
  const double gj = c->g[j];
  c->g[j + 1] = -sn * gj;
  c->g[j] = cs * gj;
  c->k = j + 1;
  c->its += 1;
  const double res = fabs(c->g[j + 1]);
  c->resid = res;
  if (!finite_d(res) || !finite_d(hn)) {
    c->nonfinite = 1;
    c->active = 0;
  } else if (res <= c->target) {
    c->converged = 1;
    c->active = 0;
  } else if (hn == 0.0) {        // lucky breakdown: the Krylov space is invariant
    c->active = 0;
  } else if (j + 1 >= c->m) {    // end of the cycle
    c->active = 0;
  } else {
    c->scale[j + 1] = 1.0 / hn;
  }
  mirror_active(c->host_active, c->active);
}

}  // namespace jfnk
