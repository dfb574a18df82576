/*
 * jfnk.h -- C ABI of libjfnk, a GB300 (sm_103a) implementation of the
 * matrix-free Jacobian-free Newton-Krylov (JFNK) hot path of
 * "Robust Matrix-Free Newton-Krylov Solvers via Automatic Differentiation".
 *
 * The method solves the discrete residual equation F(x^k, x*) = 0 (Eq. 2) by
 * Newton's method, J(x^k) dx = -F(x^k) (Eq. 4), with the relative stopping
 * test ||F(x^k)|| / ||F(x*)|| < tol_Newton (Eq. 5) and a backtracking line
 * search (Sec. 2). The Newton system is solved by a Krylov method that sees
 * the Jacobian only through Jacobian-vector products (Sec. 3.1): either the
 * forward-mode AD product jvp(F, x, v) = (F(x), J(x) v) (Eq. 9), computed
 * here by one dual-number sweep of the residual stencil, or the finite-
 * difference quotient (F(x + eps v) - F(x)) / eps (Eq. 7) with the step of
 * Eq. 8 or the scaled rule sqrt(eps_mach) (1 + ||x||) / ||v||.
 *
 * Conventions for every entry point:
 *  - Status: every function returns a jfnk_status; nothing aborts, exits or
 *    throws across the ABI. jfnk_last_error() gives the message of the last
 *    failure on a context.
 *  - Arrays: contiguous structure-of-arrays planes, field-major, then
 *    row-major (y, x): element (f, j, i) is at f * ny * nx + j * nx + i. The
 *    1D Burgers problem has ny = 1.
 *  - Ownership: array arguments are borrowed. Device pointers must stay
 *    valid until the call returns (every call below is synchronous with
 *    respect to the context's stream unless stated). Host pointers are
 *    accepted where stated; the library then copies through its own device
 *    buffers. The context owns all workspace and frees it in jfnk_destroy.
 *  - Threads: a context is used by one host thread at a time.
 */
#ifndef JFNK_H
#define JFNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Raised when an entry point, a struct layout or a documented behaviour of
 * this header changes (3: jfnk_tune; the library reads no environment). */
#define JFNK_ABI_VERSION 3
#define JFNK_MAX_RESTART 64   /* largest GMRES restart length m */

typedef struct jfnk_ctx jfnk_ctx;

typedef enum {
  JFNK_OK = 0,
  JFNK_E_INVALID = 1,        /* bad argument; nothing was done */
  JFNK_E_OOM = 2,            /* workspace would exceed the HBM budget or cudaMalloc failed */
  JFNK_E_CUDA = 3,           /* a CUDA runtime call failed; see jfnk_last_error */
  JFNK_E_NOT_CONVERGED = 4,  /* Newton reached max_newton without meeting tol_Newton */
  JFNK_E_BREAKDOWN = 5,      /* Krylov breakdown (BiCGSTAB rho, r_hat.v or omega = 0; CG p.Ap = 0) */
  JFNK_E_NONFINITE = 6,      /* a residual norm or Krylov scalar became Inf/NaN */
  JFNK_E_LINESEARCH = 7,     /* reserved: line search failures are counted, not fatal */
  JFNK_E_TIMEOUT = 8,        /* a bounded device wait expired */
  JFNK_E_BUSY = 9            /* jfnk_poll: the request is still running */
} jfnk_status;

typedef enum { JFNK_AD = 0, JFNK_FD = 1 } jfnk_linearisation;
/* Krylov solver of the Newton system J d = -F (Sec. 3): restarted GMRES,
 * BiCGSTAB, or conjugate gradients, which needs J symmetric positive definite
 * (the reaction-diffusion / Allen-Cahn implicit step with theta dt small
 * enough; not the radiation, Burgers or Maxwell Jacobians). CG applies one
 * JVP per iteration with the p.Jp dot fused into it; a non-positive or
 * non-finite p.Jp ends it with JFNK_E_BREAKDOWN. */
typedef enum { JFNK_GMRES = 0, JFNK_BICGSTAB = 1, JFNK_CG = 2 } jfnk_krylov;
typedef enum {
  JFNK_BURGERS1D = 0,     /* p[0] = nu                                              */
  JFNK_ALLEN_CAHN2D = 1,  /* p[0] = D, p[1] = coefficient of the +u term (1 or 0),
                             p[2] = 0: periodic unit square (cells of width 1/nx);
                             1: the paper's reaction-diffusion walls, u = 0 on the
                             boundary of [-1/2, 1/2]^2, unknowns on the interior
                             nodes (spacing 1/(nx + 1))                           */
  JFNK_SU_OLSON2D = 2,    /* p[0] = sigma, p[1] = a, p[2] = T_b, p[3] = rho,
                             p[4] = 1 flux limiter on / 0 off                        */
  JFNK_MAXWELL_TE2D = 3,  /* p[0] = k, p[1] = chi3; aux[0] = eps_r (nx*ny),
                             aux[1] = source (Re plane, Im plane; 2*nx*ny)           */
  JFNK_BURGERS2D = 4,     /* p[0] = nu >= 0, p[1] = side L of the periodic square
                             (0: 2 pi), p[2] = Courant number C (0: fixed dt)       */
  JFNK_MAXWELL_VEC2D = 5  /* p[0] = w > 0, p[1] = chi >= 0, p[2] = loss L >= 0 (the
                             paper's 0.05); aux[0] unused (NULL), aux[1] = current J
                             (Re Jx, Im Jx, Re Jy, Im Jy planes; 4*nx*ny)            */
} jfnk_pde;
/* JFNK_MAXWELL_VEC2D is the paper's vector TE Maxwell problem in a Kerr
 * medium (App. A, Time-Harmonic Maxwell's Equations in Kerr Media): the
 * boundary-value problem curl curl E - w^2 eps(E) E = i w J with
 * eps(E) = (1 - L i)(1 + chi |E|), |E| = sqrt(|Ex|^2 + |Ey|^2), E = (Ex, Ey)
 * on the nodes x_i = i/(nx - 1), y_j = j/(ny - 1) of the unit square, whose
 * walls are perfect electric conductors: the rows of the tangential component
 * on a wall are F = E_t, and a neighbour beyond a wall is the image across it
 * (tangential component odd, normal even). State planes [Re Ex, Im Ex, Re Ey,
 * Im Ey]; central differences of the curl-curl operator with the mixed
 * derivative on the four corner neighbours; |E| = 0 takes a zero derivative.
 * jfnk_solve starts from the Born guess (the chi = 0 problem solved from
 * zero) when opts.born_start is set; the paper's continuation over the
 * frequency w is a sequence of such solves (jfnk_set_problem per w). */
/* JFNK_BURGERS2D is the paper's 2D viscous Burgers problem (App. A, Burgers'
 * Equation): U = (u, v) on nodes x_i = i L/nx, y_j = j L/ny of the periodic
 * square, second-order central differences for the advection u D_x U +
 * v D_y U and the 5-point Laplacian for nu lap U; state [u plane, v plane].
 * With C > 0 each implicit step of jfnk_solve first sets its time step from
 * the current state by the CFL rule of that passage,
 *   dt = C min(hx / max|u|, hy / max|v|, 1 / (2 nu (1/hx^2 + 1/hy^2))),
 * a term whose denominator is zero left out (all left out: JFNK_E_INVALID);
 * the maxima are reduced on the device and prob.dt is ignored. */
typedef enum {
  JFNK_FP64 = 0,        /* everything in FP64                                                 */
  JFNK_FP32 = 1,        /* state, residual, JVP and basis in FP32 (Hessenberg in FP64)        */
  JFNK_MIXED_FP32 = 2,  /* FP64 state, residual, update, line search and Hessenberg;
                           JVP and Krylov vectors in FP32                                     */
  JFNK_MIXED_BF16 = 3   /* as MIXED_FP32 with the GMRES basis stored in BF16                  */
} jfnk_precision;
typedef enum { JFNK_EPS_SCALED = 0, JFNK_EPS_PAPER = 1 } jfnk_fd_rule;
/* Right preconditioner of GMRES for the vector Maxwell problem: the paper's
 * block-diagonal complex-shifted-Laplacian (App. A, Preconditioning), per
 * node M_xx = 2/hy^2 - w^2 eps_p, M_yy = 2/hx^2 - w^2 eps_p with
 * eps_p = eps(E)(1 - beta i) at the current Newton iterate (beta =
 * opts.precond_damping, the paper's 0.5), 1 on the rows of the tangential
 * components on the walls. GMRES solves J M^-1 y = -F (every Jacobian-vector
 * product applies M^-1 to its direction first, AD or FD) and the Newton step
 * is d = M^-1 y. Only with krylov = JFNK_GMRES and the vector Maxwell
 * problem (JFNK_E_INVALID otherwise). */
typedef enum { JFNK_PRECOND_NONE = 0, JFNK_PRECOND_CSLP = 1 } jfnk_precond;
/* Arnoldi orthogonalisation of GMRES (Sec. 3): classical Gram-Schmidt applied
 * twice, or the same two passes with the second one delayed by one Arnoldi
 * step (delayed CGS2), which fuses them into one dots pass and one update
 * pass over the basis. Same Krylov space, basis and iterates in exact
 * arithmetic; each cycle that converges before its last column applies the
 * Jacobian once more. DCGS2 runs on the streaming kernels: N (all fields) a
 * multiple of 8, else JFNK_E_INVALID. The batched entry points take CGS2 or
 * DCGS2 (any N: there the passes are phases of the batch kernel). */
/* JFNK_DCGS2_FUSED is delayed CGS2 with the update of step j, the AD JVP of
 * the next candidate and the dots of step j + 1 in one kernel, so the basis
 * is read once per step instead of twice. It needs lin = JFNK_AD, prec =
 * JFNK_FP32 or JFNK_MIXED_FP32 and a 2D problem with face neighbours only
 * (Allen-Cahn, Maxwell TE, 2D Burgers) whose rows fit its shared-memory plan
 * (JFNK_E_INVALID otherwise). It gives the iterates of JFNK_DCGS2 but is
 * slower on GB300, being bound by instruction issue rather than HBM. */
typedef enum { JFNK_CGS2 = 0, JFNK_DCGS2 = 1, JFNK_DCGS2_FUSED = 2 } jfnk_ortho;

/* One nonlinear problem: PDE, grid and time step (App. A and the benchmark
 * variants). The implicit step is the theta-method residual
 *   F(x; b) = M(x) - theta dt G(x) - b,   b = M(x^n) + (1 - theta) dt G(x^n),
 * M the identity except for the radiation problem (material energy a T^4).
 * theta = 1/2 is the paper's Crank-Nicolson; 1 is backward Euler. The
 * Maxwell problem is a boundary-value problem, F = G (dt, theta unused). */
typedef struct {
  int pde;            /* jfnk_pde */
  int nx, ny;         /* cells (nodes for JFNK_MAXWELL_VEC2D); ny = 1 for Burgers */
  double dt, theta;
  double p[8];        /* PDE parameters, see jfnk_pde */
  const double* aux[2];  /* Maxwell eps_r and source (the vector form: aux[1] = J), FP64,
                            host or device; copied by jfnk_set_problem; NULL: eps_r = 1,
                            no source */
} jfnk_problem;

typedef struct {
  int lin;            /* jfnk_linearisation */
  int krylov;         /* jfnk_krylov */
  int prec;           /* jfnk_precision */
  int restart;        /* GMRES restart length m, 1..JFNK_MAX_RESTART; 0: chosen by the library's
                         autotuner, which solves the first Newton system of a problem class
                         (PDE, grid, precision, linearisation, Arnoldi form) once with each of
                         m = 10, 20, 30, 40, 60 to tol_krylov, times them, keeps the fastest
                         that converged for that class on the context and uses its step (so
                         the choice is made at equal tolerance, not equal iterates). Only
                         jfnk_solve and the server's single-solve worker; the batched entry
                         points need m >= 1. */
  int max_newton;     /* Newton iterations per nonlinear solve */
  int max_krylov;     /* GMRES restart cycles; BiCGSTAB / CG iterations */
  double tol_newton;  /* Eq. 5 */
  double tol_krylov;  /* ||r|| <= tol_krylov ||b|| */
  int fd_rule;        /* jfnk_fd_rule */
  double fd_eps;      /* > 0: fixed FD step instead of the rule */
  double ls_c1;       /* Armijo constant: accept ||F(x+a dx)|| <= (1 - c1 a) ||F(x)|| */
  double ls_min_alpha;/* smallest trial step; accepted when no trial passes */
  int born_start;     /* Maxwell: solve the chi3 = 0 problem from zero first */
  int ortho;          /* jfnk_ortho (GMRES) */
  int precond;        /* jfnk_precond (GMRES, vector Maxwell) */
  double precond_damping;  /* beta of eps_p = eps(E)(1 - beta i); the paper's 0.5 */
} jfnk_opts;

typedef struct {
  int status;           /* jfnk_status of the last nonlinear solve */
  int steps_done;       /* implicit steps completed */
  int steps_failed;     /* steps whose final ||F||/||F0|| missed 100 x tol_newton */
  int newton_its, krylov_its, jvp_calls, ls_backtracks, ls_failures, krylov_failures;
  double res0;          /* ||F(x*)|| of the last solve (Eq. 5 denominator) */
  double res_final;     /* final ||F|| of the last solve */
  double ms;            /* host wall time of the call */
  double dt_last;       /* time step of the last implicit step (the CFL step when adaptive) */
  double ls_alpha[16];  /* jfnk_solve: the step alpha the line search accepted in each of the
                           first 16 Newton iterations of the last nonlinear solve (0: none);
                           the batched and served paths leave it 0 */
  int restart_used;     /* jfnk_solve, GMRES: the restart length of the last Krylov solve (the
                           autotuner's choice when opts.restart = 0) */
} jfnk_report;

/* Defaults of the paper for a precision (Sec. 3.3): tol_Newton 1e-6 / 1e-4,
 * tol_Krylov 1e-8 / 1e-6 (FP64 / FP32), 15 Newton iterations, 100 Krylov
 * cycles, GMRES(30) with CGS2, AD, scaled FD rule, c1 = 1e-4,
 * alpha_min = 2^-10, no preconditioner (damping 0.5 when one is chosen). */
void jfnk_default_opts(jfnk_opts* opts, int prec);

/* Create a context on CUDA device `device`. hbm_budget caps the workspace
 * the context may allocate (0: no cap). cuda_stream is a cudaStream_t to
 * issue all work on (NULL: the context creates its own non-blocking stream).
 * Returns JFNK_E_INVALID for a bad device, JFNK_E_CUDA on runtime errors. */
jfnk_status jfnk_create(jfnk_ctx** out, int device, size_t hbm_budget, void* cuda_stream);

/* Validate and install a problem; copies aux arrays. Workspace for the
 * Krylov solver is sized lazily by jfnk_solve. JFNK_E_INVALID on bad sizes
 * or parameters. */
jfnk_status jfnk_set_problem(jfnk_ctx* ctx, const jfnk_problem* prob);

/* One Jacobian-vector product of the installed residual at x along v.
 * lin = JFNK_AD: one dual-number sweep gives F(x) (written to F_out when it
 * is not NULL) and J(x) v (Eq. 9). lin = JFNK_FD: (F(x + eps v) - F(x))/eps
 * (Eq. 7) with eps = fd_eps when fd_eps > 0, else the scaled rule
 * sqrt(eps_mach)(1 + ||x||)/||v|| (both norms reduced on the device; for
 * v = 0 the rule takes ||v|| = 1, so the step stays finite and the quotient
 * is zero up to the rounding of F(x) between the two sweeps). prec =
 * JFNK_FP64: x, v, b, F_out, Jv_out are double; JFNK_FP32: float. b is the
 * constant part of the theta-method residual (NULL: zero). All pointers are
 * device pointers; the call is stream-ordered and returns after the work is
 * queued. A 2D Burgers problem with an adaptive step is refused as in
 * jfnk_residual. */
jfnk_status jfnk_jvp(jfnk_ctx* ctx, int lin, int prec, const void* x, const void* v,
                     const void* b, void* F_out, void* Jv_out, double fd_eps);

/* Residual of the installed problem: F_out = F(x; b) in precision prec
 * (device pointers, stream-ordered). A 2D Burgers problem with an adaptive
 * step (Courant number p[2] > 0) has no time step outside jfnk_solve:
 * JFNK_E_INVALID (install it with p[2] = 0 and the step as dt). */
jfnk_status jfnk_residual(jfnk_ctx* ctx, int prec, const void* x, const void* b, void* F_out);

/* Solve `steps` implicit steps from x_prev (NULL: from x_inout), writing the
 * final state to x_inout; for the Maxwell problem one nonlinear solve from
 * x_inout (or the Born start). x_prev and x_inout are FP64, host or device.
 * The backtracking line search of each Newton step is decided on the device:
 * the trial residuals F(x + alpha d) for alpha = 1, 1/2, ... down to
 * ls_min_alpha are queued together, the last block of each trial applies the
 * Armijo test and either accepts it or halves alpha for the next, and the
 * trials after the accepted one do nothing; the host reads the result back
 * once per Newton step. Synchronous. Returns JFNK_OK when every step
 * converged, otherwise the status of the first failing step; rep (host, may
 * be NULL) gets counts. */
jfnk_status jfnk_solve(jfnk_ctx* ctx, const jfnk_opts* opts, const double* x_prev,
                       double* x_inout, int steps, jfnk_report* rep);

/* Batched solves: `count` independent problems solved together, each with
 * its own options (probs[i], opts[i]) and step count (steps[i]; ignored for
 * the Maxwell problem), each exactly as jfnk_solve would define it (Newton
 * with the Armijo line search of Sec. 2, restarted GMRES with CGS2 or delayed
 * CGS2 Arnoldi of Sec. 3 (opts[i].ortho; JFNK_DCGS2_FUSED is refused), the AD JVP of Eq. 9 or the FD quotient of Eq. 7, the theta
 * method of Eq. 2, the Born start). The state of every solve lives on the
 * device; each launch of the batch kernel advances every unfinished solve by
 * one phase of that iteration (a JVP sweep, one Gram-Schmidt pass or the
 * delayed form's dots or update pass, a residual, a line-search trial ...), and the host replays a captured CUDA
 * graph of such launches until all are done, so small solves share launches
 * instead of each paying its own launch and synchronisation latency.
 * Supported: krylov = JFNK_GMRES, prec = JFNK_FP64, JFNK_FP32 or
 * JFNK_MIXED_FP32 (JFNK_E_INVALID otherwise, nothing runs). The problems do
 * not use the context's installed problem. x_prev[i] (x_prev or x_prev[i]
 * may be NULL: start from x_inout[i]) and x_inout[i] are FP64 host or device
 * arrays of the problem's size; results are written to x_inout[i].
 * Reductions are summed in a fixed order over 256-cell units of each
 * problem, so a problem's result does not depend on the other problems of
 * the batch, on the tile size or on the grid (it differs from jfnk_solve's
 * at rounding level). reps[i] (may be NULL) gets each solve's counts,
 * statuses[i] (may be NULL) its status as jfnk_solve would return it.
 * Synchronous. Returns the first non-OK status in index order, JFNK_E_OOM
 * when the summed workspace exceeds the context's HBM budget. */
jfnk_status jfnk_solve_batch(jfnk_ctx* ctx, int count, const jfnk_problem* probs, const jfnk_opts* opts,
                             const double* const* x_prev, double* const* x_inout, const int* steps,
                             jfnk_report* reps, int* statuses);

/* Batch engine counters: kernel launches issued by jfnk_solve_batch (and the
 * batched part of the server) so far, and the tile size (cells) the
 * autotuner chose for problems of this PDE, precision and grid (0: none yet). */
jfnk_status jfnk_batch_stats(jfnk_ctx* ctx, long long* kernel_launches, int* tile_cells, int pde, int prec,
                             int nx, int ny);

/* Tuning and diagnostic switches of a context; each call sets one knob.
 *   JFNK_TUNE_BATCH_TILE: value > 0 fixes the batch engine's cells per tile
 *     (rounded down to a multiple of 256, clamped to 256..2048) for every
 *     problem class jfnk_solve_batch has not tuned yet on this context; 0
 *     restores the measured choice per class. Results do not depend on it.
 *   JFNK_TUNE_BULK_COPY: 1 (the default) lets the single-solve path stream the
 *     Krylov basis through the bulk-copy ring; 0 restricts it to the plain-load
 *     passes (classical Gram-Schmidt only: the delayed forms then return
 *     JFNK_E_INVALID, as on grids the ring cannot take).
 * JFNK_E_INVALID (nothing changes) for a NULL context, an unknown knob or a
 * value outside its range. Call between solves: a solve in flight on another
 * thread may see either setting. */
typedef enum { JFNK_TUNE_BATCH_TILE = 0, JFNK_TUNE_BULK_COPY = 1 } jfnk_tune_knob;
jfnk_status jfnk_tune(jfnk_ctx* ctx, int knob, long long value);

/* Serving: queue a solve of `prob` (steps as in jfnk_solve) and return a
 * ticket at once. x0 and x_out are FP64 host or device arrays that must stay
 * valid until jfnk_poll returns a final status for the ticket. Requests are
 * admitted when their workspace fits the context's HBM budget. Requests up
 * to 2^20 unknowns (all fields) go to the batch engine, where every admitted
 * request advances in the same launches; larger ones run one at a time on a
 * single solve worker, concurrently with the batch engine. */
jfnk_status jfnk_submit(jfnk_ctx* ctx, const jfnk_problem* prob, const jfnk_opts* opts,
                        const double* x0, double* x_out, int steps, unsigned long long* ticket);

/* JFNK_E_BUSY while the request runs; otherwise its final status, with rep
 * (may be NULL) filled in. Unknown tickets give JFNK_E_INVALID. */
jfnk_status jfnk_poll(jfnk_ctx* ctx, unsigned long long ticket, jfnk_report* rep);

/* Per-kernel timing: when enabled, each kernel class launched by the
 * context is bracketed by CUDA events on the context's stream and its
 * device time accumulated. jfnk_kernel_stats fills, for kernel class i,
 * names[i] (static strings), launches[i], total_ms[i] and bytes[i] (the
 * algorithmic bytes those launches had to move) for up to cap classes and
 * returns the number of classes. Reset clears the counters. */
jfnk_status jfnk_set_timing(jfnk_ctx* ctx, int enable);
int jfnk_kernel_stats(jfnk_ctx* ctx, const char** names, long long* launches,
                      double* total_ms, double* bytes, int cap);
void jfnk_reset_stats(jfnk_ctx* ctx);

/* FD Jacobian-vector product for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment convenience. Some
 * callers cannot call cudaMalloc -- code whose device memory belongs to
 * another allocator or pool, or hot paths that must never reach the driver's
 * allocator -- and jfnk_jvp needs a context whose workspace is allocated.
 * This entry point needs no context and allocates nothing: it computes
 * F(x) and (F(x + eps v) - F(x)) / eps like jfnk_jvp with lin = JFNK_FD,
 * taking its workspace (the two norms of the step rule and, when F_out is
 * NULL, F(x)) from one fixed device array that the library holds on every
 * GPU it is loaded on, until the process exits
 * (JFNK_NOALLOC_SCRATCH_BYTES).
 *   prob      host struct as for jfnk_set_problem; for the Maxwell problem
 *             aux[0] (eps_r) and aux[1] (source) are FP64 device pointers
 *             (or NULL) used in place, and prec must be JFNK_FP64.
 *   prec      JFNK_FP64 (double arrays) or JFNK_FP32 (float arrays).
 *   x, v, b   device arrays of N = nf * nx * ny entries (b may be NULL).
 *   F_out     device array for F(x), or NULL to keep F(x) in the scratch;
 *             with NULL, N * sizeof(element) must not exceed
 *             JFNK_NOALLOC_MAX_FX_BYTES, else JFNK_E_OOM and nothing runs.
 *   Jv_out    device array for the quotient.
 *   fd_eps    > 0: the step; otherwise sqrt(eps_mach)(1 + ||x||)/||v||.
 *   cuda_stream  stream for all work (NULL: the legacy default stream).
 * Errors: JFNK_E_INVALID for bad arguments, JFNK_E_OOM as above,
 * JFNK_E_CUDA when a launch fails. Stream-ordered; returns once queued.
 * The first call on each device looks the scratch array's address up for
 * that device (with it current) and keeps it for the life of the process;
 * make that first call before capturing the stream. A device reset
 * (cudaDeviceReset) unloads the array, and the kept address is then stale:
 * do not call this entry point on a device after resetting it. For v = 0 the
 * step rule takes ||v|| = 1, as in jfnk_jvp. A 2D Burgers
 * problem with an adaptive step (p[2] > 0) is JFNK_E_INVALID, as for
 * jfnk_jvp. Every call reuses the same array and clears the part that must
 * start at zero, so calls that overlap on the GPU (other streams, other host
 * threads) race on it: serialise them. */
#define JFNK_NOALLOC_MAX_FX_BYTES 4194304u
#define JFNK_NOALLOC_SCRATCH_BYTES (4352u + JFNK_NOALLOC_MAX_FX_BYTES)
jfnk_status jfnk_jvp_fd_noalloc(const jfnk_problem* prob, int prec, const void* x, const void* v, const void* b,
                                void* F_out, void* Jv_out, double fd_eps, void* cuda_stream);

const char* jfnk_last_error(const jfnk_ctx* ctx);
const char* jfnk_status_string(int status);
void jfnk_destroy(jfnk_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* JFNK_H */
