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
  volatile int* host_active;       // mapped host words (may be null): [0] mirrors `active`, [1] the
                                   // delayed-CGS2 steps completed in this cycle (dcgs_after_update)
  // arrays
  double H[(kMaxM + 1) * kMaxM];   // Hessenberg, column-major H[j * (kMaxM + 1) + i], rotated in place
  double h1[kMaxM + 1];            // first Gram-Schmidt pass of column j
  double h2[kMaxM + 1];            // second pass
  double cs[kMaxM], sn[kMaxM];     // Givens rotations
  double g[kMaxM + 1];             // rotated right-hand side beta e_1
  double y[kMaxM];                 // least-squares solution at the end of a cycle
  double scale[kMaxM + 1];         // v_t = scale[t] u_t
  // delayed CGS2 (dcgs_step): completed columns before rotation, the first
  // projection of the newest column, and the coefficients of the update pass
  double Hraw[(kMaxM + 1) * kMaxM];
  double hprev[kMaxM + 1];
  double da[kMaxM + 1];            // q_j = dgamma u_j - sum_i da[i] q_i
  double dc[kMaxM + 1];            // u_{j+1} = dinvr (w - sum_i dc[i] q_i - dc[j] q_j)
  double dgamma, dinvr;
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

// Backtracking line search of one Newton step (Sec. 2, after Eq. 4), decided
// on the device. The host queues the trial residuals F(x + alpha d) for
// alpha = 1, 1/2, ... down to the smallest trial at once; the last block of
// each trial applies the Armijo test to its ||F|| and either accepts the
// trial (done = 1: the trials queued after it return at once, so the trial
// buffers keep the accepted state) or halves alpha for the next one. The
// smallest trial is accepted when no trial passes (a line-search failure).
struct LsCtl {
  double fnorm;       // ||F(x_k)||, the merit of the current iterate
  double alpha;       // step of the next trial
  double c1, min_alpha;
  double ft;          // ||F(x_k + alpha d)|| of the accepted trial
  double alpha_acc;   // the accepted step
  int done;           // a trial has been accepted
  int backtracks;     // halvings in this Newton step
  int failures;       // 1 when the smallest trial was taken without passing
  int accept_first;   // take the first trial as it is (the linear Born solve)
};

__device__ __forceinline__ void ls_decide(LsCtl* c, double f2) {
  const double ft = sqrt(f2), a = c->alpha;
  bool accept = c->accept_first || (isfinite(ft) && ft <= (1.0 - c->c1 * a) * c->fnorm);
  if (!accept && a * 0.5 < c->min_alpha) {
    accept = true;
    c->failures = 1;
  }
  if (accept) {
    c->ft = ft;
    c->alpha_acc = a;
    c->done = 1;
  } else {
    c->alpha = a * 0.5;
    c->backtracks += 1;
  }
}

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

// gmres_givens_step run by every thread of a block: the column and the
// previous rotations are staged in shared memory first, so thread 0's
// sequential rotation reads shared memory instead of making one L2 round trip
// per entry. Same arithmetic in the same order.
__device__ __forceinline__ void gmres_givens_step_block(GmresCtl* c, int j, double n2) {
  __shared__ double s_col[kMaxM + 1], s_cs[kMaxM], s_sn[kMaxM];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    s_col[i] = c->h1[i] + c->h2[i];
    if (i < j) { s_cs[i] = c->cs[i]; s_sn[i] = c->sn[i]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* col = c->H + (size_t)j * (kMaxM + 1);
    const double hn = sqrt(n2);
    s_col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = s_col[i], b = s_col[i + 1];
      s_col[i] = s_cs[i] * a + s_sn[i] * b;
      s_col[i + 1] = -s_sn[i] * a + s_cs[i] * b;
    }
    const double f = s_col[j], gg = s_col[j + 1];
    const double r = hypot(f, gg);
    double cs = 1.0, sn = 0.0;
    if (r != 0.0) { cs = f / r; sn = gg / r; }
    c->cs[j] = cs;
    c->sn[j] = sn;
    s_col[j] = cs * f + sn * gg;
    s_col[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; ++i) col[i] = s_col[i];
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
    } else if (hn == 0.0) {
      c->active = 0;
    } else if (j + 1 >= c->m) {
      c->active = 0;
    } else {
      c->scale[j + 1] = 1.0 / hn;
    }
    mirror_active(c->host_active, c->active);
  }
}

// Delayed CGS2 (the second Gram-Schmidt pass of each Arnoldi vector one step
// late), step j, run by every thread of one block after the fused dots pass.
// Slot j of the basis holds the candidate u_j (projected once, not
// normalised); the JVP was applied to ut = sigma u_j, sigma = scale[j], giving
// w. S holds the pass's sums: S[2i] = q_i . u_j, S[2i+1] = q_i . w for i < j,
// S[2j] = u_j . u_j, S[2j+1] = u_j . w (has_w = 0: the last step of a cycle,
// no w). With s = sigma S[2i], rho^2 = sigma^2 S[2j] - s.s:
//   * column j-1 is completed: H[:j, j-1] = hprev + s / sigma,
//     H[j, j-1] = rho / sigma, then rotated and tested as in CGS2;
//   * q_j = (ut - Q s) / rho, and the first projection of A q_j follows from
//     w through the completed columns: z = H[:j+1, :j] s,
//     h_i = (t_i - z_i) / rho (i < j), h_j = ((sigma S[2j+1] - s.t) / rho - z_j) / rho;
//   * the update pass forms q_j and u_{j+1} = A q_j - Q_{j+1} h from the
//     coefficients da, dc, dgamma, dinvr.
// Everything the step reads is in shared memory: the caller stages the sums
// S and the scalars, dcgs_stage stages the rest (the completed columns into
// `hs`, which must hold j (kMaxM + 1) doubles) in the same round of loads, so
// the sequential part makes no global round trips; sums over i are warp
// butterflies, quotients are products with one reciprocal. sh must hold
// 5 (kMaxM + 1) doubles.
__device__ __forceinline__ void dcgs_stage(GmresCtl* c, int j, double* sh, double* hs) {
  constexpr int LD = kMaxM + 1;
  double* col = sh + 2 * LD;
  const int cj = j - 1;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    col[i] = c->hprev[i];
    if (i < cj) { sh[3 * LD + i] = c->cs[i]; sh[4 * LD + i] = c->sn[i]; }
  }
  const int ne = (j > 0 ? cj : 0) * LD;
  for (int e0 = threadIdx.x; e0 < ne; e0 += 8 * blockDim.x) {   // eight loads in flight per thread
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * (int)blockDim.x;
      v[q] = e < ne ? __ldcg(&c->Hraw[e]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * (int)blockDim.x;
      if (e < ne) hs[e] = v[q];
    }
  }
}

// GB300 issues a warp's FP64 instruction over many cycles (two FP64 FMAs per
// clock per SM), so each scalar is formed once, by one thread, and the
// rotation chain carries one FMA per step; isig = 1 / sigma comes from the
// caller, formed while the tail's loads are in flight.
__device__ __forceinline__ void dcgs_step(GmresCtl* c, int j, const double* S, bool has_w, double* sh, double* hs,
                                          double sigma, double isig, double g_prev, double target, int m,
                                          int active0, int its0) {
  constexpr int LD = kMaxM + 1;
  double* ss = sh;             // s
  double* zz = sh + LD;        // z
  double* col = sh + 2 * LD;   // column j-1: completed, then rotated
  const double* s_cs = sh + 3 * LD;
  const double* s_sn = sh + 4 * LD;
  __shared__ int s_go, s_bad;
  __shared__ double s_s2, s_st, s_rho, s_irs, s_hn;
  __shared__ double s_cb[kMaxM + 1], s_sb[kMaxM + 1], s_a[kMaxM + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cj = j - 1;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const double si = sigma * S[2 * i];
    ss[i] = si;
    col[i] += si * isig;
  }
  __syncthreads();
  if (warp == 0) {
    double v = 0.0;
    for (int i = lane; i < j; i += 32) v += ss[i] * ss[i];
    v = warp_sum(v);
    if (lane == 0) s_s2 = v;
  } else if (warp == 1) {
    double v = 0.0;
    for (int i = lane; i < j; i += 32) v += ss[i] * S[2 * i + 1];
    v = warp_sum(v);
    if (lane == 0) s_st = v;
  }
  __syncthreads();
  // thread 0: rho (one rsqrt for rho and its reciprocal) and H[j, j-1]
  if (threadIdx.x == 0) {
    const double alpha = sigma * sigma * S[2 * j];
    const double rho2 = alpha - s_s2;
    const double irs = rho2 > 0.0 ? rsqrt(rho2) : 0.0;
    s_irs = irs;
    s_rho = rho2 * irs;
    s_hn = s_rho * isig;
    s_bad = !finite_d(rho2) || !finite_d(sigma);
  }
  __syncthreads();
  const double rho = s_rho, irs = s_irs, hn = s_hn;
  const bool bad = s_bad != 0;
  // the completed (unrotated) column j-1 into hs, and the products of the
  // rotation chain that do not depend on the carried entry
  if (j > 0 && !bad) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) hs[(size_t)cj * LD + i] = col[i];
    if (threadIdx.x == 0) {
      hs[(size_t)cj * LD + j] = hn;
      col[j] = hn;
    }
    for (int i = threadIdx.x; i < cj; i += blockDim.x) {
      const double b = (i + 1 < j) ? col[i + 1] : hn;
      s_cb[i] = s_cs[i] * b;
      s_sb[i] = s_sn[i] * b;
    }
  }
  __syncthreads();
  if (warp == 0) {
    // rotation of column j-1, the residual estimate and the cycle's flags; the
    // other warps meanwhile form z, which needs only the unrotated columns
    if (lane == 0) {
      int active = active0;
      int go = 1;
      if (bad) {
        c->nonfinite = 1;
        active = 0;
        go = 0;
      } else if (j == 0) {
        c->g[0] = g_prev * rho;      // r = beta rho q_0
      } else {
        // the carried entry a_{i+1} = -sn_i a_i + cs_i b_i: one dependent FMA per
        // rotation (the products cs_i b_i were formed above by all threads); the
        // rotated entries cs_i a_i + sn_i b_i are formed from s_a afterwards
        double a = col[0];
        for (int i = 0; i < cj; ++i) {
          s_a[i] = a;
          a = fma(-s_sn[i], a, s_cb[i]);
        }
        const double f = a, gg = col[cj + 1];
        const double r2 = fma(f, f, gg * gg);     // Hessenberg entries: no overflow in the squares
        double cs = 1.0, sn = 0.0;
        if (r2 != 0.0) { const double ir = rsqrt(r2); cs = f * ir; sn = gg * ir; }
        c->cs[cj] = cs;
        c->sn[cj] = sn;
        col[cj] = cs * f + sn * gg;
        col[cj + 1] = 0.0;
        const double g1 = -sn * g_prev;
        c->g[cj + 1] = g1;
        c->g[cj] = cs * g_prev;
        c->k = j;
        c->its = its0 + 1;                   // its0 staged with the other scalars: no load on this path
        const double res = fabs(g1);
        c->resid = res;
        if (!finite_d(res) || !finite_d(hn)) {
          c->nonfinite = 1;
          active = 0;
        } else if (res <= target) {
          c->converged = 1;
          active = 0;
        } else if (hn == 0.0 || j >= m) {   // lucky breakdown, or the end of the cycle
          active = 0;
        }
        if (!active) go = 0;
      }
      if (go && has_w && rho == 0.0 && active) {   // the candidate vanished: nothing left to project
        active = 0;
        go = 0;
      }
      if (!has_w) go = 0;
      if (!active) {
        c->active = 0;
        mirror_active(c->host_active, 0);
      }
      s_go = go;
    }
  } else if (!bad && has_w && rho != 0.0) {
    // z = H[:j+1, :j] s over the completed (unrotated) columns, upper Hessenberg:
    // one thread per row, a sequential FMA chain (few FP64 operations, so the
    // rotation that warp 0 runs meanwhile keeps the FP64 pipe)
    const int i = (int)threadIdx.x - 32;
    if (i <= j) {
      double z = 0.0;
      for (int l = (i > 0 ? i - 1 : 0); l < j; ++l) z = fma(hs[(size_t)l * LD + i], ss[l], z);
      zz[i] = z;
    }
  }
  __syncthreads();
  // the completed column j-1 (unrotated and rotated) back to global memory;
  // rotated entries below the new rotation from the carried entries
  if (j > 0 && !bad)
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      c->Hraw[(size_t)cj * LD + i] = hs[(size_t)cj * LD + i];
      c->H[(size_t)cj * LD + i] = i < cj ? fma(s_cs[i], s_a[i], s_sb[i]) : col[i];
    }
  if (!s_go) return;
  const double irho = irs;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const double h = (S[2 * i + 1] - zz[i]) * irho;
    c->hprev[i] = h;
    c->da[i] = ss[i] * irho;
    c->dc[i] = zz[i] + rho * h;
  }
  if (threadIdx.x == 0) {
    const double qw = (sigma * S[2 * j + 1] - s_st) * irho;
    const double h = (qw - zz[j]) * irho;
    c->hprev[j] = h;
    c->dc[j] = zz[j] + rho * h;
    c->dgamma = sigma * irho;
    c->dinvr = irho;
  }
}

// After the update pass of step j: q_j is stored normalised, u_{j+1} has
// squared norm n2.
__device__ __forceinline__ void dcgs_after_update(GmresCtl* c, int j, double n2) {
  c->scale[j] = 1.0;
  if (!finite_d(n2)) {
    c->nonfinite = 1;
    c->active = 0;
    mirror_active(c->host_active, 0);
  } else {
    c->scale[j + 1] = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  }
  if (c->host_active) {   // step j done: the host's lookahead bound, without a stream event
    c->host_active[1] = j + 1;
    __threadfence_system();
  }
}

}  // namespace jfnk
