// batch.h -- many independent Newton-GMRES solves advanced together.
//
// Each solve keeps its whole Newton / line-search / restarted-GMRES control
// state on the device (BatState) and moves through the phases below. One
// launch of the batch kernel advances every unfinished solve by exactly one
// phase: the solve's cells are cut into tiles, a persistent grid takes tiles
// from a shared work counter, and the last tile of a solve to finish performs
// the solve's scalar step (reduction, Givens rotation, Newton test, line-search
// decision) and sets its next phase. No host round trip sits between phases,
// so the host replays a captured CUDA graph of many launches.
//
// Reductions are summed per unit of kBatUnit cells, then over units in order,
// so results do not depend on the tile size, on the grid or on which other
// solves share the launch. Internal; not part of the C ABI.
#pragma once

#include "ctl.cuh"
#include "kernels.h"

namespace jfnk {

constexpr int kBatThreads = 256;   // threads per CTA
constexpr int kBatUnit = 256;      // cells per reduction unit
constexpr int kBatPart = 136;      // partial sums kept per unit (>= 2 (kMaxM + 1): delayed-CGS2 dots)

enum BatPhase {
  PH_IN = 0,     // state <- caller's initial value (zero for the Born stage)
  PH_CFL,        // adaptive time step: max|u|, max|v| -> CFL rule (2D Burgers with C > 0)
  PH_RHS,        // b = M(x^n) + (1 - theta) dt G(x^n)
  PH_RES,        // F(x), ||F||^2, ||x||^2 (and the FP32 copy of x)
  PH_FX32,       // F(x) in FP32 for the FD quotient of a mixed-precision solve
  PH_GINIT,      // u_0 = -F, rhs = -F, d = 0, beta = ||F||
  PH_JVP,        // w = J v_j
  PH_A1,         // h1 = V^T w
  PH_A2,         // w -= V h1; h2 = V^T w
  PH_A3,         // w -= V h2; u_{j+1} = w; ||w||^2 -> Givens step
  PH_GUPD,       // d += V y
  PH_RJVP,       // restart: u_0 = rhs - J d, ||u_0||^2
  PH_LS,         // trial x + alpha d: F, ||F||^2, ||x + alpha d||^2 -> Armijo test
  PH_D1,         // delayed CGS2: q_i . u_j, q_i . w (i <= j) -> the coefficient step (whole CTA)
  PH_D2,         // delayed CGS2: q_j -> slot j, u_{j+1} -> slot j + 1, ||u_{j+1}||^2
  PH_OUT,        // caller's result <- state
  PH_DONE
};

struct BatState {
  int phase, cur, step, newton_it, cycle, j, stage, fresh;
  unsigned int arrive;             // tiles of the current phase that have finished
  int status, first_bad;
  int steps_done, steps_failed, newton_its, krylov_its, jvp_calls, ls_backtracks, ls_failures, krylov_failures;
  int pad_;
  double fn2, fnorm, f0, alpha, dn2, res0, res_final;
  double xn2[2];                   // ||x||^2 of the two state buffers
  double dt, thdt, c_old;          // time step of the current implicit step, theta dt, (1 - theta) dt
  GmresCtl g;
};

struct BatDesc {
  ProbDev P;
  long long N;                     // unknowns nf * ncell
  int tc, ntile, nunit;            // cells per tile, tiles, reduction units
  int ts, tj;                      // state and JVP / basis precision (VT_F64, VT_F32)
  int lin, fd_rule, m, max_newton, max_krylov, steps, born;
  int ortho;                       // JFNK_CGS2 (phases A1-A3) or JFNK_DCGS2 (phases D1-D2)
  double tol_newton, tol_krylov, fd_eps, ls_c1, ls_min_alpha;
  void* x[2]; void* F[2]; float* x32[2];
  void* b; float* b32; float* F32;
  void* d;                         // Newton step (state precision)
  void* rhs;                       // -F in the JVP precision
  void* w;                         // Arnoldi work vector
  void* V;                         // basis, (m + 1) x N, unnormalised columns u_t
  double* part;                    // nunit x kBatPart partial sums
  double* io;                      // FP64 initial state in, result out
  BatState* st;
  int* done_flag;                  // set to 1 when the solve reaches PH_DONE
};

struct BatLaunch {
  const BatDesc* desc;
  const int2* items;               // (solve, tile)
  int nitems;
  unsigned int* next;              // work counter (zero between launches)
  unsigned int* ndone;             // CTAs finished (zero between launches)
};

// One launch of the batch kernel for the solves of one (PDE, ts, tj) group.
cudaError_t batch_launch(int pde, int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st);
// Largest useful grid of that kernel (resident CTAs on all SMs).
int batch_grid_cap(int pde, int ts, int tj, int nsm);

cudaError_t batch_launch_burgers(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st);
cudaError_t batch_launch_allen_cahn(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st);
cudaError_t batch_launch_su_olson(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st);
cudaError_t batch_launch_maxwell(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st);
cudaError_t batch_launch_burgers2d(int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st);
int batch_occ_burgers(int ts, int tj);
int batch_occ_allen_cahn(int ts, int tj);
int batch_occ_su_olson(int ts, int tj);
int batch_occ_maxwell(int ts, int tj);
int batch_occ_burgers2d(int ts, int tj);

}  // namespace jfnk
