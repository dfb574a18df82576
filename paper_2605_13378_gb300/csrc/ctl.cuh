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
  // the inputs of the next step by step parity (step j reads slot j & 1): the
  // deferred form runs step j in every block of the update pass while block 0
  // writes its outputs, so what the step overwrites (hprev, g[j-1], its) is
  // read from these copies
  double hprev_p[2][kMaxM + 1];
  double gprev_p[2];
  int its_p[2];
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
    c->gprev_p[0] = beta;
    c->its_p[0] = c->its;
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
// late), step j, run after the fused dots pass of step j: by its last block,
// or (the deferred form) by every block of the update pass at its start, block
// 0 alone writing the control state.
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

// The threads that run a step together: a whole block (the dots pass's last
// block, the fused pass), or the consumer warps 1.. of the update pass, which
// run it while warp 0 keeps filling the ring (named barrier 1).
struct BlockTeam {
  __device__ int rank() const { return (int)threadIdx.x; }
  __device__ int size() const { return (int)blockDim.x; }
  __device__ void sync() const { __syncthreads(); }
};
struct ConsumerTeam {
  __device__ int rank() const { return (int)threadIdx.x - 32; }
  __device__ int size() const { return (int)blockDim.x - 32; }
  __device__ void sync() const { asm volatile("bar.sync 1, %0;" ::"r"((int)blockDim.x - 32) : "memory"); }
};

// GB300 issues a warp's FP64 instruction over many cycles (two FP64 FMAs per
// clock per SM), so each scalar is formed once, by one thread, and the
// rotation chain carries one FMA per step; isig = 1 / sigma comes from the
// caller, formed while the tail's loads are in flight.
//
// kStagedH: the completed columns 0..j-2 are staged in `hs` (j (kMaxM + 1)
// doubles; the new column j-1 is added there) and each row of z is one
// sequential chain. Otherwise they are read from global memory, `hs` holds
// only the new column (kMaxM + 1 doubles), and each row of z is split over
// two or four threads of a warp with a fixed combining order.
// Only the `writer` updates the control state (the rotation, H, Hraw, the
// cycle's flags and the next step's inputs, also by step parity); every
// caller gets the update pass's coefficients in o_da, o_dc, o_gamma, o_invr
// (rounded to O: the control state's FP64, or the update pass's accumulator).
// Returns whether the update pass of step j runs (every thread of the team).
template <class Team, bool kStagedH, class O>
__device__ __forceinline__ bool dcgs_step_t(GmresCtl* c, int j, const double* S, bool has_w, double* sh, double* hs,
                                            double sigma, double isig, double g_prev, double target, int m,
                                            int active0, int its0, Team tm, bool writer, O* o_da, O* o_dc,
                                            O* o_gamma, O* o_invr) {
  constexpr int LD = kMaxM + 1;
  double* ss = sh;             // s
  double* zz = sh + LD;        // z
  double* col = sh + 2 * LD;   // column j-1: completed, then rotated
  const double* s_cs = sh + 3 * LD;
  const double* s_sn = sh + 4 * LD;
  __shared__ int s_go, s_bad;
  __shared__ double s_s2, s_st, s_rho, s_irs, s_hn;
  __shared__ double s_cb[kMaxM + 1], s_sb[kMaxM + 1], s_a[kMaxM + 1];
  const int r = tm.rank(), T = tm.size();
  const int lane = r & 31, warp = r >> 5;
  const int cj = j - 1, nxt = (j + 1) & 1;
  double* hnew = kStagedH ? hs + (size_t)(j > 0 ? cj : 0) * LD : hs;   // the completed column j-1, unrotated
  for (int i = r; i < j; i += T) {
    const double si = sigma * S[2 * i];
    ss[i] = si;
    col[i] += si * isig;
  }
  tm.sync();
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
  tm.sync();
  // one thread: rho (one rsqrt for rho and its reciprocal) and H[j, j-1]
  if (r == 0) {
    const double alpha = sigma * sigma * S[2 * j];
    const double rho2 = alpha - s_s2;
    const double irs = rho2 > 0.0 ? rsqrt(rho2) : 0.0;
    s_irs = irs;
    s_rho = rho2 * irs;
    s_hn = s_rho * isig;
    s_bad = !finite_d(rho2) || !finite_d(sigma);
  }
  tm.sync();
  const double rho = s_rho, irs = s_irs, hn = s_hn;
  const bool bad = s_bad != 0;
  // the completed (unrotated) column j-1 into hnew, and the products of the
  // rotation chain that do not depend on the carried entry
  if (j > 0 && !bad) {
    for (int i = r; i < j; i += T) hnew[i] = col[i];
    if (r == 0) {
      hnew[j] = hn;
      col[j] = hn;
    }
    for (int i = r; i < cj; i += T) {
      const double b = (i + 1 < j) ? col[i + 1] : hn;
      s_cb[i] = s_cs[i] * b;
      s_sb[i] = s_sn[i] * b;
    }
  }
  tm.sync();
  if (warp == 0) {
    // rotation of column j-1, the residual estimate and the cycle's flags; the
    // other warps meanwhile form z, which needs only the unrotated columns
    if (lane == 0) {
      int active = active0;
      int go = 1;
      if (bad) {
        if (writer) c->nonfinite = 1;
        active = 0;
        go = 0;
      } else if (j == 0) {
        const double g0 = g_prev * rho;   // r = beta rho q_0
        if (writer) {
          c->g[0] = g0;
          c->gprev_p[nxt] = g0;
          c->its_p[nxt] = its0;
        }
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
        col[cj] = cs * f + sn * gg;
        col[cj + 1] = 0.0;
        const double g1 = -sn * g_prev;
        const double res = fabs(g1);
        if (writer) {
          c->cs[cj] = cs;
          c->sn[cj] = sn;
          c->g[cj + 1] = g1;
          c->g[cj] = cs * g_prev;
          c->k = j;
          c->its = its0 + 1;                 // its0 staged with the other scalars: no load on this path
          c->resid = res;
          c->gprev_p[nxt] = g1;
          c->its_p[nxt] = its0 + 1;
        }
        if (!finite_d(res) || !finite_d(hn)) {
          if (writer) c->nonfinite = 1;
          active = 0;
        } else if (res <= target) {
          if (writer) c->converged = 1;
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
      if (!active && writer) {
        c->active = 0;
        mirror_active(c->host_active, 0);
      }
      s_go = go;
    }
  } else if (!bad && has_w && rho != 0.0) {
    // z = H[:j+1, :j] s over the completed (unrotated) columns, upper Hessenberg
    // (few FP64 operations, so the rotation that warp 0 runs meanwhile keeps the
    // FP64 pipe)
    if constexpr (kStagedH) {
      // one thread per row, a sequential FMA chain
      const int i = r - 32;
      if (i <= j) {
        double z = 0.0;
        for (int l = (i > 0 ? i - 1 : 0); l < j; ++l) z = fma(hs[(size_t)l * LD + i], ss[l], z);
        zz[i] = z;
      }
    } else {
      // P threads per row (the lanes of a row are adjacent in one warp), each
      // taking every P-th completed column from global memory with eight loads in
      // flight; the partial chains are combined by butterflies, then the newest
      // column's term is added
      const int P = (j + 1) * 4 <= T - 32 ? 4 : 2;
      const int i = (r - 32) / P, q = (r - 32) - i * P;
      double z = 0.0;
      if (i <= j && j > 0) {
        int l = (i > 0 ? i - 1 : 0) + q;
        for (; l + 7 * P < cj; l += 8 * P) {
          double h[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) h[u] = __ldcg(&c->Hraw[(size_t)(l + u * P) * LD + i]);
#pragma unroll
          for (int u = 0; u < 8; ++u) z = fma(h[u], ss[l + u * P], z);
        }
        for (; l < cj; l += P) z = fma(__ldcg(&c->Hraw[(size_t)l * LD + i]), ss[l], z);
      }
      z += __shfl_xor_sync(0xffffffffu, z, 1);
      if (P == 4) z += __shfl_xor_sync(0xffffffffu, z, 2);
      if (q == 0 && i <= j) zz[i] = j > 0 ? fma(hnew[i], ss[cj], z) : 0.0;
    }
  }
  tm.sync();
  // the completed column j-1 (unrotated and rotated) back to global memory;
  // rotated entries below the new rotation from the carried entries
  if (writer && j > 0 && !bad)
    for (int i = r; i <= j; i += T) {
      c->Hraw[(size_t)cj * LD + i] = hnew[i];
      c->H[(size_t)cj * LD + i] = i < cj ? fma(s_cs[i], s_a[i], s_sb[i]) : col[i];
    }
  const bool go = s_go != 0;
  if (!go) return false;
  const double irho = irs;
  for (int i = r; i < j; i += T) {
    const double h = (S[2 * i + 1] - zz[i]) * irho;
    if (writer) {
      c->hprev[i] = h;
      c->hprev_p[nxt][i] = h;
    }
    o_da[i] = (O)(ss[i] * irho);
    o_dc[i] = (O)(zz[i] + rho * h);
  }
  if (r == 0) {
    const double qw = (sigma * S[2 * j + 1] - s_st) * irho;
    const double h = (qw - zz[j]) * irho;
    if (writer) {
      c->hprev[j] = h;
      c->hprev_p[nxt][j] = h;
    }
    o_dc[j] = (O)(zz[j] + rho * h);
    *o_gamma = (O)(sigma * irho);
    *o_invr = (O)irho;
  }
  return true;
}

__device__ __forceinline__ void dcgs_step(GmresCtl* c, int j, const double* S, bool has_w, double* sh, double* hs,
                                          double sigma, double isig, double g_prev, double target, int m,
                                          int active0, int its0) {
  dcgs_step_t<BlockTeam, true, double>(c, j, S, has_w, sh, hs, sigma, isig, g_prev, target, m, active0, its0, BlockTeam{},
                               true, c->da, c->dc, &c->dgamma, &c->dinvr);
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
