// jfnk.cu -- the C ABI of libjfnk: contexts, problems, the Newton driver with
// backtracking line search (Sec. 2, Eqs. 4-5), the host side of restarted
// GMRES and BiCGSTAB (Sec. 3.1), time stepping, per-kernel timing.
//
// All arithmetic runs in the kernels of stencil.cu and krylov.cu; the host
// only sequences launches on the context's stream and reads back a few
// scalars (Newton residual norms, the Krylov control block after each GMRES
// cycle). Inside a cycle the Arnoldi steps are launched back to back; the
// device clears an `active` flag (mirrored into mapped host memory) when the
// cycle converges, later launches of the cycle return at once, and the host
// stops issuing steps when it sees the flag, at most kLookahead steps late.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "batch_engine.h"
#include "jfnk.h"
#include "kernels.h"
#include "krylov.h"
#include "serve.h"

using namespace jfnk;

namespace {

enum KClass {
  KC_RESIDUAL, KC_RHS, KC_JVP_AD, KC_JVP_FD, KC_ARN1, KC_ARN2, KC_ARN3, KC_GINIT, KC_GFIN, KC_CAST,
  KC_VDOTS, KC_BICG, KC_DCGS1, KC_DCGS2, KC_CFL, KC_DCGSF, KC_COUNT
};
const char* kKClassNames[KC_COUNT] = {
    "residual", "rhs", "jvp_ad", "jvp_fd", "arnoldi_dots", "arnoldi_update_dots", "arnoldi_update_norm_givens",
    "gmres_init", "gmres_backsolve_update", "cast", "vdots", "bicgstab_vector", "arnoldi_dcgs_dots",
    "arnoldi_dcgs_update", "cfl_dt", "arnoldi_dcgs_fused"};

constexpr int kLookahead = 3;   // Arnoldi / BiCGSTAB steps the host may run ahead of the device
constexpr int kServeSlotWorkers = 1;   // single-solve workers of the request server (jfnk_submit)

// GMRES restart lengths the autotuner (opts.restart = 0) times on the first
// Newton system of a problem class
constexpr int kTuneRestarts[] = {10, 20, 30, 40, 60};
constexpr int kTuneMaxRestart = 60;
typedef std::tuple<int, int, int, int, int, int> TuneKey;   // pde, nx, ny, precision, linearisation, ortho

struct Pending {
  int cls;
  double bytes;
  int ev;       // index of the start event; stop is ev + 1
  int tag;      // iteration index inside the current Krylov loop, -1 for unconditional launches
};

struct Timer {
  bool on = false;
  long long total_launches = 0;   // every kernel launched by the solver, timed or not
  std::vector<cudaEvent_t> pool;
  int used = 0;
  std::vector<Pending> pending;
  long long launches[KC_COUNT] = {0};
  double ms[KC_COUNT] = {0};
  double bytes[KC_COUNT] = {0};
};

int prec_types(int prec, int* ts, int* tj, int* tb) {
  switch (prec) {
    case JFNK_FP64: *ts = VT_F64; *tj = VT_F64; *tb = VT_F64; return 1;
    case JFNK_FP32: *ts = VT_F32; *tj = VT_F32; *tb = VT_F32; return 1;
    case JFNK_MIXED_FP32: *ts = VT_F64; *tj = VT_F32; *tb = VT_F32; return 1;
    case JFNK_MIXED_BF16: *ts = VT_F64; *tj = VT_F32; *tb = VT_BF16; return 1;
  }
  return 0;
}

}  // namespace

struct jfnk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0, allocated = 0;
  std::string err;
  bool have_prob = false;
  jfnk_problem prob;
  ProbDev P;
  long long N = 0;
  // problem data owned by the context
  double* eps64 = nullptr; float* eps32 = nullptr;
  double* src64 = nullptr; float* src32 = nullptr;
  // small permanent device state
  double* dsc = nullptr;          // scalar slots
  unsigned int* derr = nullptr;   // device error word (bounded waits that expired)
  int nsm = 0;                    // multiprocessors: grid of the streaming kernels
  bool stream_ok = true;          // bulk-copy streaming of the basis allowed (JFNK_TUNE_BULK_COPY)
  int batch_tile = 0;             // JFNK_TUNE_BATCH_TILE: fixed cells per tile of the batch engine (0: measured)
  GmresCtl* gctl = nullptr;
  BicgCtl* bctl = nullptr;
  LsCtl* lsc = nullptr;           // line search of the current Newton step
  RedWs red{};
  int red_cap_blocks = 0;
  // pinned / mapped host memory
  volatile int* hflag = nullptr;  // mapped: [0] mirror of the Krylov `active` flag, [1] delayed-CGS2 steps done
  int* hflag_dev = nullptr;       // its device address
  double* hbuf = nullptr;         // pinned read-back buffer (16 KB)
  cudaEvent_t iter_ev[kLookahead + 1] = {};
  // workspace
  struct Ws {
    long long N = 0; int prec = -1, m = 0, krylov = -1; bool ok = false;
    void *x = nullptr, *xt = nullptr, *xn = nullptr, *F = nullptr, *Ft = nullptr, *b = nullptr, *d = nullptr;
    void *x32 = nullptr, *x32t = nullptr, *F32 = nullptr, *b32 = nullptr;
    void *rhsk = nullptr, *w = nullptr, *dj = nullptr, *V = nullptr, *dbest = nullptr;
    void *u2[2] = {nullptr, nullptr}, *w2 = nullptr;   // fused delayed-CGS2 pass: candidates, second w
    void *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
    void* user = nullptr;        // FP64 staging of user arrays
    std::vector<void*> all;
    size_t bytes = 0;
  } ws;
  void* jscratch = nullptr;       // F(x) for jfnk_jvp's FD quotient when F_out is null
  size_t jscratch_bytes = 0;
  Timer tm;
  std::map<TuneKey, int> tuned_restart;   // restart length chosen per problem class (opts.restart = 0)
  jfnk::Server* server = nullptr;
  jfnk::BatchEngine* batch = nullptr;   // jfnk_solve_batch
};

namespace {

jfnk_status fail(jfnk_ctx* c, jfnk_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

jfnk_status cuda_fail(jfnk_ctx* c, cudaError_t e, const char* where) {
  return fail(c, JFNK_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

jfnk_status dalloc(jfnk_ctx* ctx, void** p, size_t bytes, std::vector<void*>* track) {
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->allocated + bytes > ctx->budget)
    return fail(ctx, JFNK_E_OOM, "workspace of " + std::to_string(ctx->allocated + bytes) +
                                     " bytes exceeds the HBM budget of " + std::to_string(ctx->budget));
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, JFNK_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->allocated += bytes;
  if (track) track->push_back(*p);
  return JFNK_OK;
}

void ws_free(jfnk_ctx* ctx) {
  for (void* p : ctx->ws.all) cudaFree(p);
  ctx->allocated -= ctx->ws.bytes;
  ctx->ws = jfnk_ctx::Ws();
}

// --------------------------------------------------------------------------
// timing
// --------------------------------------------------------------------------
int tm_begin(jfnk_ctx* ctx, int cls, double bytes, int tag, int nkernels = 1) {
  Timer& t = ctx->tm;
  t.total_launches += nkernels;
  if (!t.on) return -1;
  if (t.used + 2 > (int)t.pool.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return -1; }
      t.pool.push_back(e);
    }
  }
  const int ev = t.used;
  t.used += 2;
  cudaEventRecord(t.pool[ev], ctx->stream);
  t.pending.push_back(Pending{cls, bytes, ev, tag});
  return ev;
}
void tm_end(jfnk_ctx* ctx, int ev) {
  if (ev < 0) return;
  cudaEventRecord(ctx->tm.pool[ev + 1], ctx->stream);
}
// After a stream synchronisation: accumulate every pending launch whose tag
// is below `valid` (launches of iterations the device skipped are dropped).
void tm_harvest(jfnk_ctx* ctx, int valid, double fin_bytes) {
  Timer& t = ctx->tm;
  if (!t.on) return;
  for (const Pending& p : t.pending) {
    if (p.tag == -2 || (p.tag >= 0 && p.tag >= valid)) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.pool[p.ev], t.pool[p.ev + 1]) != cudaSuccess) { cudaGetLastError(); continue; }
    t.launches[p.cls] += 1;
    t.ms[p.cls] += ms;
    t.bytes[p.cls] += (p.cls == KC_GFIN && fin_bytes >= 0) ? fin_bytes : p.bytes;
  }
  t.pending.clear();
  t.used = 0;
}

// --------------------------------------------------------------------------
// workspace
// --------------------------------------------------------------------------
jfnk_status ensure_ws(jfnk_ctx* ctx, int prec, int m, int krylov) {
  jfnk_ctx::Ws& w = ctx->ws;
  if (w.ok && w.N == ctx->N && w.prec == prec && w.krylov == krylov && (krylov != JFNK_GMRES || w.m >= m))
    return JFNK_OK;
  cudaStreamSynchronize(ctx->stream);
  ws_free(ctx);
  int ts, tj, tb;
  prec_types(prec, &ts, &tj, &tb);
  const long long N = ctx->N;
  const size_t ss = vt_size(ts), sj = vt_size(tj), sb = vt_size(tb);
  size_t before = ctx->allocated;
  std::vector<void*>* tr = &w.all;
  jfnk_status s;
#define AL(ptr, nbytes) if ((s = dalloc(ctx, &(ptr), (nbytes), tr)) != JFNK_OK) { w.bytes = ctx->allocated - before; ws_free(ctx); return s; }
  AL(w.x, N * ss); AL(w.xt, N * ss); AL(w.xn, N * ss); AL(w.F, N * ss); AL(w.Ft, N * ss); AL(w.b, N * ss);
  AL(w.d, N * ss);
  AL(w.user, N * 8);
  if (tj != ts) { AL(w.x32, N * sj); AL(w.x32t, N * sj); AL(w.F32, N * sj); AL(w.b32, N * sj); }
  AL(w.rhsk, N * sj); AL(w.w, N * sj); AL(w.dj, N * sj);
  if (krylov == JFNK_GMRES) {
    AL(w.V, (size_t)(m + 1) * N * sb);
    AL(w.dbest, N * ss);   // the restart autotuner's best step so far
    if (tj == VT_F32 && tb == VT_F32) { AL(w.u2[0], N * sj); AL(w.u2[1], N * sj); AL(w.w2, N * sj); }
  } else {
    AL(w.r, N * sj); AL(w.rhat, N * sj); AL(w.p, N * sj); AL(w.v, N * sj); AL(w.s, N * sj); AL(w.t, N * sj);
  }
#undef AL
  w.bytes = ctx->allocated - before;
  w.N = N; w.prec = prec; w.m = m; w.krylov = krylov; w.ok = true;
  return JFNK_OK;
}

jfnk_status ensure_red(jfnk_ctx* ctx) {
  int need = vec_blocks(ctx->N);
  if (2 * ctx->nsm > need) need = 2 * ctx->nsm;   // grid of the streaming kernels, and the deferred
                                                  // delayed-CGS2 partials after its own kMaxK per block
  if (ctx->have_prob) {
    const StencilGeom g = stencil_geom(ctx->P);
    if (g.max_blocks > need) need = g.max_blocks;
  }
  if (need <= ctx->red_cap_blocks) return JFNK_OK;
  if (ctx->red.partials) { cudaFree(ctx->red.partials); ctx->allocated -= (size_t)ctx->red_cap_blocks * kMaxK * 8; }
  ctx->red.partials = nullptr;
  jfnk_status s = dalloc(ctx, &ctx->red.partials, (size_t)need * kMaxK * 8, nullptr);
  if (s != JFNK_OK) { ctx->red_cap_blocks = 0; return s; }
  ctx->red_cap_blocks = need;
  ctx->red.max_blocks = need;
  return JFNK_OK;
}

// --------------------------------------------------------------------------
// the solver for one context and precision
// --------------------------------------------------------------------------
struct Solver {
  jfnk_ctx* ctx;
  jfnk_opts o;
  int ts, tj, tb, td;
  long long N;
  ProbDev P;
  // current / trial buffers (swapped on accepted line-search steps)
  void *x, *xt, *F, *Ft, *x32, *x32t;
  double *sc, *st;    // [||F||^2, ||x||^2] of the current and of the trial state
  jfnk_report rep;

  size_t ss() const { return vt_size(ts); }
  size_t sj() const { return vt_size(tj); }
  size_t sb() const { return vt_size(tb); }
  double aux_bytes(int tcode) const { return (P.pde == 3 && P.eps64) ? (double)P.ncell * vt_size(tcode) : 0.0; }

  jfnk_status residual(const void* xx, const void* dd, double alpha, void* Fo, void* xo, void* x32o, double* sums,
                       int tcode, const void* bb, LsCtl* ls = nullptr, int tag = -1) {
    double bytes = (double)N * vt_size(tcode) * (1 + (dd ? 1 : 0) + (bb ? 1 : 0) + (Fo ? 1 : 0) + (xo ? 1 : 0)) +
                   (x32o ? (double)N * 4 : 0.0) + aux_bytes(tcode);
    int ev = tm_begin(ctx, KC_RESIDUAL, bytes, tag);
    cudaError_t e = launch_residual(P, tcode, xx, dd, alpha, bb, Fo, xo, (float*)x32o, ctx->red, sums, ctx->stream,
                                    ls);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "residual kernel");
    return JFNK_OK;
  }

  jfnk_status jvp(JvpArgs& a, int tag) {
    a.t = tj;
    a.err = ctx->derr;
    if (a.precond && a.lin == 1 && o.fd_eps <= 0 && o.fd_rule == JFNK_EPS_SCALED) {
      // the FD step of the preconditioned direction: ||M^-1 v|| in place of ||v|| (times the vector's scale)
      cudaError_t e = launch_precond(P, tj, a.x, a.v, nullptr, ctx->dsc + 18, o.precond_damping, ctx->red,
                                     ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "preconditioner norm kernel");
      a.vn2 = ctx->dsc + 18;
    }
    const double s = (double)sj();
    double bytes = (double)N * (s + vt_size(a.tv) + s) + aux_bytes(tj);     // x, v -> out
    if (a.lin == 1) bytes += (double)N * s;                                 // F(x)
    if (a.add) bytes += (double)N * s;
    for (int k = 0; k < a.ndots; ++k) if (a.dw[k]) bytes += (double)N * s;
    int ev = tm_begin(ctx, a.lin == 0 ? KC_JVP_AD : KC_JVP_FD, bytes, tag);
    cudaError_t e = launch_jvp(P, a, ctx->red, ctx->stream);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "jvp kernel");
    return JFNK_OK;
  }

  JvpArgs jvp_base() {
    JvpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.lin = o.lin;
    a.t = tj;
    a.tv = tj;
    a.x = (tj == ts) ? x : x32;
    a.b = (tj == ts) ? ctx->ws.b : ctx->ws.b32;
    a.Fx = (tj == ts) ? F : ctx->ws.F32;
    if (P.bvp) a.b = nullptr;
    a.c_jv = 1.0;
    a.eps_fixed = o.fd_eps;
    a.eps_rule = o.fd_rule;
    a.xn2 = sc + 1;
    a.precond = o.precond == JFNK_PRECOND_CSLP ? 1 : 0;
    a.pbeta = o.precond_damping;
    return a;
  }

  // ---- the Newton step from the right-preconditioned solve: d = M^-1 y (in place)
  jfnk_status precond_solution() {
    if (o.precond != JFNK_PRECOND_CSLP) return JFNK_OK;
    cudaError_t e = launch_precond(P, td, x, ctx->ws.d, ctx->ws.d, nullptr, o.precond_damping, ctx->red, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "preconditioner kernel");
    return JFNK_OK;
  }

  jfnk_status cast(int ti, int to, const void* src, void* dst, double c) {
    int ev = tm_begin(ctx, KC_CAST, (double)N * (vt_size(ti) + vt_size(to)), -1);
    cudaError_t e = launch_cast(ti, to, N, src, dst, c, ctx->stream);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cast kernel");
    return JFNK_OK;
  }

  jfnk_status sync_read(const void* dev, size_t bytes) {
    CK(cudaMemcpyAsync(ctx->hbuf, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream), "read-back");
    CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    return JFNK_OK;
  }

  // ---- adaptive time step (2D Burgers CFL rule) from the current state x;
  // *dt gets the step (NaN when the state is not finite) -----------------
  jfnk_status cfl_step(double* dt) {
    const int ev = tm_begin(ctx, KC_CFL, (double)N * vt_size(ts), -1);
    cudaError_t e = launch_cfl_dt(P, ts, x, ctx->dsc + 16, ctx->red, ctx->nsm, ctx->stream);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cfl kernel");
    jfnk_status s = sync_read(ctx->dsc + 16, sizeof(double));
    if (s) return s;
    *dt = ctx->hbuf[0];
    if (std::isinf(*dt)) return fail(ctx, JFNK_E_INVALID, "CFL step undefined: nu = 0 and the state is at rest");
    if (std::isfinite(*dt)) set_dt(&P, *dt);
    return JFNK_OK;
  }

  // ---- wait until the device has completed `steps` delayed-CGS2 steps of the
  // current cycle (mapped word host_active[1]) or stopped the cycle (word 0
  // cleared). Bounded: after 2 s without either the host drains the stream,
  // which always ends because every device wait is itself bounded.
  jfnk_status wait_progress(int steps) {
    const auto t0 = std::chrono::steady_clock::now();
    for (long long spin = 0; ctx->hflag[1] < steps && ctx->hflag[0] != 0; ++spin) {
      if ((spin & 1023) == 1023 && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(2)) {
        CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
        break;
      }
    }
    return JFNK_OK;
  }

  // ---- one cycle of delayed-CGS2 Arnoldi: candidate u_j in basis slot j,
  // JVP, fused dots (completes column j - 1), fused update (q_j, u_{j+1});
  // the dots of u_m complete the last column. The device clears `active`
  // when the cycle stops; kernels queued past that point return at once.
  // Without per-kernel timing the three kernels of a step are launched
  // programmatically (PDL, stream.cuh), each dispatched while the one before
  // it drains, and the host bounds its lookahead by the mapped word that the
  // update pass advances (GmresCtl::host_active[1]) instead of by a stream
  // event, which would sit between two kernels and serialise them.
  jfnk_status dcgs_cycle(int m, int* steps_run) {
    jfnk_ctx::Ws& w = ctx->ws;
    const double nv = (double)N;
    const bool pdl = !ctx->tm.on;
    ctx->hflag[1] = 0;
    int j = 0;
    for (; j < m; ++j) {
      if (j >= kLookahead) {
        if (pdl) {
          jfnk_status s = wait_progress(j - kLookahead + 1);
          if (s) return s;
        } else {
          CK(cudaEventSynchronize(ctx->iter_ev[(j - kLookahead) % (kLookahead + 1)]), "iteration event");
        }
      }
      if (*ctx->hflag == 0) break;
      JvpArgs a = jvp_base();
      a.v = (const char*)w.V + (size_t)j * N * sb();
      a.tv = tb;
      a.vscale = ctx->gctl->scale + j;
      a.out = w.w;
      a.active = &ctx->gctl->active;
      a.pdl = pdl ? 1 : 0;   // after the update pass (or a kernel launched plainly): neither writes x
      jfnk_status s = jvp(a, j);
      if (s) return s;
      const double bs = (double)(j + 1) * nv * sb();
      int ev1 = tm_begin(ctx, KC_DCGS1, bs + nv * sj(), j);
      // the coefficient step of step j runs at the start of its update pass (deferred form)
      cudaError_t e = launch_dcgs(1, tb, tj, N, w.V, j, w.w, ctx->gctl, ctx->red, ctx->derr, ctx->nsm, ctx->stream,
                                  pdl, true);
      tm_end(ctx, ev1);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "dcgs dots kernel");
      int ev2 = tm_begin(ctx, KC_DCGS2, bs + nv * sj() + 2.0 * nv * sb(), j + 1);   // did work iff j < k
      e = launch_dcgs(2, tb, tj, N, w.V, j, w.w, ctx->gctl, ctx->red, ctx->derr, ctx->nsm, ctx->stream, pdl, true);
      tm_end(ctx, ev2);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "dcgs update kernel");
      if (!pdl) CK(cudaEventRecord(ctx->iter_ev[j % (kLookahead + 1)], ctx->stream), "event record");
    }
    if (j == m) {   // the last column of the cycle
      int ev1 = tm_begin(ctx, KC_DCGS1, (double)(m + 1) * nv * sb(), m);
      cudaError_t e = launch_dcgs(1, tb, tj, N, w.V, m, nullptr, ctx->gctl, ctx->red, ctx->derr, ctx->nsm,
                                  ctx->stream, !ctx->tm.on);
      tm_end(ctx, ev1);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "dcgs dots kernel");
    }
    *steps_run = j;
    return JFNK_OK;
  }

  // ---- the same cycle with one pass per step (dcgs_fused.cuh): JVP and dots
  // of u_0 as above, then per step j the update of step j, the JVP of
  // u_{j+1} and the dots of step j + 1 in one kernel; the pass of step m - 1
  // takes the dots of u_m without a JVP and so completes the last column.
  // Candidates alternate between two buffers, and so do the JVP outputs.
  // Chosen by opts.ortho = JFNK_DCGS2_FUSED (validate_opts checks that it
  // applies): it reads the basis once per step instead of twice, but with one
  // column per thread per row it is bound by instruction issue and latency,
  // and the two streaming passes are faster on GB300.
  jfnk_status dcgs_cycle_fused(int m, int* steps_run) {
    jfnk_ctx::Ws& w = ctx->ws;
    const double nv = (double)N;
    void* U[2] = {w.u2[0], w.u2[1]};
    void* W[2] = {w.w, w.w2};
    {
      JvpArgs a = jvp_base();
      a.v = w.V;
      a.tv = tb;
      a.vscale = ctx->gctl->scale;
      a.out = W[0];
      a.active = &ctx->gctl->active;
      jfnk_status s = jvp(a, 0);
      if (s) return s;
      int ev1 = tm_begin(ctx, KC_DCGS1, nv * sb() + nv * sj(), 0);
      cudaError_t e = launch_dcgs(1, tb, tj, N, w.V, 0, W[0], ctx->gctl, ctx->red, ctx->derr, ctx->nsm, ctx->stream);
      tm_end(ctx, ev1);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "dcgs dots kernel");
      CK(cudaMemcpyAsync(U[0], w.V, (size_t)N * sj(), cudaMemcpyDeviceToDevice, ctx->stream), "copy u_0");
    }
    const void* X = (tj == ts) ? x : x32;
    const double aux = (P.pde == 3 && P.eps64) ? (double)P.ncell * 4.0 : 0.0;
    int j = 0;
    for (; j < m; ++j) {
      if (j >= kLookahead) {
        CK(cudaEventSynchronize(ctx->iter_ev[(j - kLookahead) % (kLookahead + 1)]), "iteration event");
      }
      if (*ctx->hflag == 0) break;
      const bool has_w = j + 1 < m;
      // reads slots 0..j-1, u_j, w_j (and x); writes q_j, u_{j+1} (and J u_{j+1})
      const double bytes = ((double)j + 4.0 + (has_w ? 2.0 : 0.0)) * nv * sb() + (has_w ? aux : 0.0);
      int ev = tm_begin(ctx, KC_DCGSF, bytes, j + 1);
      cudaError_t e = launch_dcgs_fused(P, N, w.V, j, has_w, j == 0, U[j & 1], U[(j + 1) & 1], W[j & 1],
                                        W[(j + 1) & 1], X, ctx->gctl, ctx->red, ctx->derr, ctx->nsm, ctx->stream);
      tm_end(ctx, ev);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "fused dcgs kernel");
      CK(cudaEventRecord(ctx->iter_ev[j % (kLookahead + 1)], ctx->stream), "event record");
    }
    *steps_run = j;
    return JFNK_OK;
  }

  // ---- restarted GMRES(m): J d = -F ------------------------------------
  jfnk_status gmres(int* kstatus) {
    jfnk_ctx::Ws& w = ctx->ws;
    const int m = o.restart;
    rep.restart_used = m;
    const double nv = (double)N;
    const bool streamed = ctx->stream_ok && stream_supported(N);
    const bool fused = o.ortho == JFNK_DCGS2_FUSED;
    *ctx->hflag = 1;   // before any launch that may clear it
    int ev = tm_begin(ctx, KC_GINIT, nv * (ss() + sb() + sj() + ss()), -1);
    cudaError_t e = launch_gmres_init(ts, tj, tb, td, N, F, w.V, w.rhsk, w.d, ctx->gctl, sc, o.tol_krylov, m,
                                      ctx->stream);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gmres init");
    *kstatus = 0;
    for (int cycle = 0; cycle < o.max_krylov; ++cycle) {
      if (cycle > 0) {
        *ctx->hflag = 1;
        // restart: u_0 = r = rhs - J d, beta = ||r||
        const void* dv = w.d;
        if (td != tj) {
          jfnk_status s = cast(td, tj, w.d, w.dj, 1.0);
          if (s) return s;
          dv = w.dj;
        }
        JvpArgs a = jvp_base();
        a.v = dv;
        a.out = (tb == tj) ? w.V : w.w;
        a.c_jv = -1.0;
        a.add = w.rhsk;
        a.c_add = 1.0;
        a.ndots = 1;
        a.sums = ctx->dsc + 8;
        a.post = POST_GMRES_RESTART;
        a.post_arg = ctx->gctl;
        if (o.lin == 1 && o.fd_eps <= 0 && o.fd_rule == JFNK_EPS_SCALED) {
          const void* aa[3] = {dv, nullptr, nullptr};
          const void* bb[3] = {nullptr, nullptr, nullptr};
          int ev2 = tm_begin(ctx, KC_VDOTS, nv * sj(), -1);
          e = launch_vdots(tj, N, 1, aa, bb, ctx->dsc + 10, ctx->red, nullptr, ctx->stream);
          tm_end(ctx, ev2);
          if (e != cudaSuccess) return cuda_fail(ctx, e, "norm kernel");
          a.vn2 = ctx->dsc + 10;
        }
        jfnk_status s = jvp(a, -1);
        if (s) return s;
        if (tb != tj) {
          s = cast(tj, tb, w.w, w.V, 1.0);
          if (s) return s;
        }
      }
      if (o.ortho == JFNK_DCGS2 || o.ortho == JFNK_DCGS2_FUSED) {
        int steps_run = 0;
        jfnk_status s = fused ? dcgs_cycle_fused(m, &steps_run) : dcgs_cycle(m, &steps_run);
        if (s) return s;
        e = cudaSuccess;
        if (steps_run > 0) {
          int ev4 = tm_begin(ctx, KC_GFIN, 0.0, -1, 2);
          e = launch_gmres_finish(tb, td, N, w.V, w.d, ctx->gctl, steps_run, ctx->stream, 1, ctx->derr, ctx->nsm);
          tm_end(ctx, ev4);
          if (e != cudaSuccess) return cuda_fail(ctx, e, "gmres update");
        }
        CK(cudaMemcpyAsync((char*)ctx->hbuf + 8192, ctx->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream),
           "read-back");
        s = sync_read(ctx->gctl, kGmresHeadBytes);
        if (s) return s;
        GmresCtl head;
        std::memcpy(&head, ctx->hbuf, kGmresHeadBytes);
        unsigned derr = 0;
        std::memcpy(&derr, (char*)ctx->hbuf + 8192, sizeof(unsigned));
        if (derr) return fail(ctx, JFNK_E_TIMEOUT, "a bounded wait on a bulk copy expired in the Arnoldi kernels");
        tm_harvest(ctx, head.k + 1, (double)head.k * nv * sb() + 2.0 * nv * vt_size(td));
        // JVPs of the cycle: one per candidate, u_0 .. u_k (u_k only when the cycle stopped before its end)
        rep.jvp_calls += (head.k < m ? head.k + 1 : m) + (cycle > 0 ? 1 : 0);
        if (head.nonfinite) { rep.krylov_its += head.its; *kstatus = JFNK_E_NONFINITE; return JFNK_OK; }
        if (head.converged) { rep.krylov_its += head.its; return JFNK_OK; }
        if (cycle == o.max_krylov - 1) { rep.krylov_its += head.its; *kstatus = JFNK_E_NOT_CONVERGED; return JFNK_OK; }
        continue;
      }
      int launched = 0;
      for (int j = 0; j < m; ++j) {
        if (j >= kLookahead) {
          CK(cudaEventSynchronize(ctx->iter_ev[(j - kLookahead) % (kLookahead + 1)]), "iteration event");
        }
        if (*ctx->hflag == 0) break;
        const int k = j + 1;
        JvpArgs a = jvp_base();
        a.v = (const char*)w.V + (size_t)j * N * sb();
        a.tv = tb;
        a.vscale = ctx->gctl->scale + j;
        a.out = w.w;
        a.active = &ctx->gctl->active;
        jfnk_status s = jvp(a, j);
        if (s) return s;
        const double bs = (double)k * nv * sb();
        for (int pass = 1; pass <= 3; ++pass) {
          const double bytes = bs + nv * sj() * (pass == 2 ? 2 : 1) + (pass == 3 ? nv * sb() : 0.0);
          int ev3 = tm_begin(ctx, KC_ARN1 + pass - 1, bytes, j);
          if (streamed)
            e = launch_basis_stream(pass, tb, tj, td, N, w.V, k, k, w.w, nullptr, ctx->gctl, ctx->red, ctx->derr,
                                    ctx->nsm, ctx->stream);
          else
            e = launch_arnoldi_pass(pass, tb, tj, N, w.V, k, w.w, ctx->gctl, ctx->red, ctx->stream);
          tm_end(ctx, ev3);
          if (e != cudaSuccess) return cuda_fail(ctx, e, "arnoldi kernel");
        }
        CK(cudaEventRecord(ctx->iter_ev[j % (kLookahead + 1)], ctx->stream), "event record");
        launched = k;
      }
      if (launched > 0) {
        int ev4 = tm_begin(ctx, KC_GFIN, 0.0, -1, 2);
        e = launch_gmres_finish(tb, td, N, w.V, w.d, ctx->gctl, launched, ctx->stream, streamed ? 1 : 0, ctx->derr,
                                ctx->nsm);
        tm_end(ctx, ev4);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "gmres update");
      }
      CK(cudaMemcpyAsync((char*)ctx->hbuf + 8192, ctx->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream),
         "read-back");
      jfnk_status s = sync_read(ctx->gctl, kGmresHeadBytes);
      if (s) return s;
      GmresCtl head;
      std::memcpy(&head, ctx->hbuf, kGmresHeadBytes);
      unsigned derr = 0;
      std::memcpy(&derr, (char*)ctx->hbuf + 8192, sizeof(unsigned));
      if (derr) return fail(ctx, JFNK_E_TIMEOUT, "a bounded wait on a bulk copy expired in the Arnoldi kernels");
      tm_harvest(ctx, head.k, (double)head.k * nv * sb() + 2.0 * nv * vt_size(td));
      rep.jvp_calls += head.k + (cycle > 0 ? 1 : 0);
      if (head.nonfinite) { rep.krylov_its += head.its; *kstatus = JFNK_E_NONFINITE; return JFNK_OK; }
      if (head.converged) { rep.krylov_its += head.its; return JFNK_OK; }
      if (cycle == o.max_krylov - 1) { rep.krylov_its += head.its; *kstatus = JFNK_E_NOT_CONVERGED; return JFNK_OK; }
    }
    return JFNK_OK;
  }

  // ---- GMRES with the restart length of the options, or -- opts.restart = 0 --
  // the one the autotuner chose for this problem class. The first Newton system
  // of a class is solved once per candidate length (kTuneRestarts), each to the
  // requested tolerance, timed on the host around the synchronous cycles; the
  // fastest candidate that converged (else the one with the smallest residual)
  // is kept for the class on this context, and its step is used.
  jfnk_status gmres_auto(int* kstatus) {
    if (o.restart > 0 || o.krylov != JFNK_GMRES) return gmres(kstatus);
    const TuneKey key{P.pde, P.nx, P.ny, o.prec, o.lin, o.ortho};
    auto it = ctx->tuned_restart.find(key);
    if (it != ctx->tuned_restart.end()) {
      o.restart = it->second;
      jfnk_status s = gmres(kstatus);
      o.restart = 0;
      return s;
    }
    int best_m = 0, best_st = 0;
    double best_t = 0.0, best_res = 0.0;
    for (int m : kTuneRestarts) {
      o.restart = m;
      const auto t0 = std::chrono::steady_clock::now();
      int kst = 0;
      jfnk_status s = gmres(&kst);
      o.restart = 0;
      if (s) return s;
      const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      GmresCtl head;
      std::memcpy(&head, ctx->hbuf, kGmresHeadBytes);   // the head of the candidate's last cycle
      const bool conv = kst == 0, best_conv = best_m > 0 && best_st == 0;
      const bool better = best_m == 0 || (conv && (!best_conv || t < best_t)) ||
                          (!conv && !best_conv && head.resid < best_res);
      if (better) {
        best_m = m; best_st = kst; best_t = t; best_res = head.resid;
        CK(cudaMemcpyAsync(ctx->ws.dbest, ctx->ws.d, (size_t)N * ss(), cudaMemcpyDeviceToDevice, ctx->stream),
           "keep step");
      }
      if (kst == JFNK_E_NONFINITE) break;
    }
    CK(cudaMemcpyAsync(ctx->ws.d, ctx->ws.dbest, (size_t)N * ss(), cudaMemcpyDeviceToDevice, ctx->stream),
       "best step");
    ctx->tuned_restart[key] = best_m;
    rep.restart_used = best_m;
    *kstatus = best_st;
    return JFNK_OK;
  }

  // ---- BiCGSTAB: J d = -F ------------------------------------------------
  jfnk_status bicgstab(int* kstatus) {
    jfnk_ctx::Ws& w = ctx->ws;
    BicgVecs vv;
    vv.F = F; vv.r = w.r; vv.rhat = w.rhat; vv.p = w.p; vv.v = w.v; vv.s = w.s; vv.t = w.t; vv.d = w.d;
    vv.sums = sc; vv.pn2 = ctx->dsc + 12; vv.sn2 = ctx->dsc + 13;
    const double nv = (double)N, s_ = (double)sj();
    const bool fd_norms = (o.lin == 1 && o.fd_eps <= 0 && o.fd_rule == JFNK_EPS_SCALED);
    *ctx->hflag = 1;
    int ev = tm_begin(ctx, KC_BICG, nv * (ss() + 5 * s_ + ss()), -1);
    cudaError_t e = launch_bicg(0, ts, tj, td, N, vv, ctx->bctl, ctx->red, 0, o.tol_krylov, ctx->stream);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bicgstab init");
    *kstatus = 0;
    for (int it = 0; it < o.max_krylov; ++it) {
      if (it >= kLookahead) {
        CK(cudaEventSynchronize(ctx->iter_ev[(it - kLookahead) % (kLookahead + 1)]), "iteration event");
      }
      if (*ctx->hflag == 0) break;
      int e1 = tm_begin(ctx, KC_BICG, nv * 4 * s_, it);
      e = launch_bicg(1, ts, tj, td, N, vv, ctx->bctl, ctx->red, it, o.tol_krylov, ctx->stream);
      tm_end(ctx, e1);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "bicgstab p");
      JvpArgs a = jvp_base();
      a.v = w.p; a.out = w.v; a.ndots = 1; a.dw[0] = w.rhat; a.sums = ctx->bctl->sums;
      a.active = &ctx->bctl->active;
      if (fd_norms) a.vn2 = vv.pn2;
      jfnk_status s = jvp(a, it);
      if (s) return s;
      int e2 = tm_begin(ctx, KC_BICG, nv * 3 * s_, it);
      e = launch_bicg(2, ts, tj, td, N, vv, ctx->bctl, ctx->red, it, o.tol_krylov, ctx->stream);
      tm_end(ctx, e2);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "bicgstab s");
      int e4 = tm_begin(ctx, KC_BICG, 0.0, -2);
      e = launch_bicg(3, ts, tj, td, N, vv, ctx->bctl, ctx->red, it, o.tol_krylov, ctx->stream);
      tm_end(ctx, e4);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "bicgstab half");
      JvpArgs b2 = jvp_base();
      b2.v = w.s; b2.out = w.t; b2.ndots = 2; b2.dw[0] = w.s; b2.dw[1] = nullptr; b2.sums = ctx->bctl->sums;
      b2.active = &ctx->bctl->active;
      if (fd_norms) b2.vn2 = vv.sn2;
      s = jvp(b2, it);
      if (s) return s;
      int e3 = tm_begin(ctx, KC_BICG, nv * (5 * s_ + 2 * ss()), it);
      e = launch_bicg(4, ts, tj, td, N, vv, ctx->bctl, ctx->red, it, o.tol_krylov, ctx->stream);
      tm_end(ctx, e3);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "bicgstab x");
      CK(cudaEventRecord(ctx->iter_ev[it % (kLookahead + 1)], ctx->stream), "event record");
    }
    jfnk_status s = sync_read(ctx->bctl, sizeof(BicgCtl));
    if (s) return s;
    BicgCtl c;
    std::memcpy(&c, ctx->hbuf, sizeof(BicgCtl));
    tm_harvest(ctx, c.its, -1.0);
    rep.krylov_its += c.its;
    rep.jvp_calls += 2 * c.its - (c.flag_half ? 1 : 0);
    if (c.nonfinite) *kstatus = JFNK_E_NONFINITE;
    else if (c.breakdown) *kstatus = JFNK_E_BREAKDOWN;
    else if (!c.converged) *kstatus = JFNK_E_NOT_CONVERGED;
    return JFNK_OK;
  }

  // ---- conjugate gradients: J d = -F (J symmetric positive definite) ----
  jfnk_status cg(int* kstatus) {
    jfnk_ctx::Ws& w = ctx->ws;
    BicgVecs vv;
    vv.F = F; vv.r = w.r; vv.rhat = nullptr; vv.p = w.p; vv.v = w.v; vv.s = nullptr; vv.t = nullptr; vv.d = w.d;
    vv.sums = sc; vv.sn2 = nullptr;
    const double nv = (double)N, s_ = (double)sj();
    const bool fd_norms = (o.lin == 1 && o.fd_eps <= 0 && o.fd_rule == JFNK_EPS_SCALED);
    vv.pn2 = fd_norms ? ctx->dsc + 12 : nullptr;
    *ctx->hflag = 1;
    int ev = tm_begin(ctx, KC_BICG, nv * (ss() + 2 * s_ + ss()), -1);
    cudaError_t e = launch_cg(0, ts, tj, td, N, vv, ctx->bctl, ctx->red, 0, o.tol_krylov, ctx->stream);
    tm_end(ctx, ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cg init");
    *kstatus = 0;
    for (int it = 0; it < o.max_krylov; ++it) {
      if (it >= kLookahead) {
        CK(cudaEventSynchronize(ctx->iter_ev[(it - kLookahead) % (kLookahead + 1)]), "iteration event");
      }
      if (*ctx->hflag == 0) break;
      if (it > 0) {
        int e1 = tm_begin(ctx, KC_BICG, nv * 3 * s_, it);
        e = launch_cg(1, ts, tj, td, N, vv, ctx->bctl, ctx->red, it, o.tol_krylov, ctx->stream);
        tm_end(ctx, e1);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cg p");
      }
      JvpArgs a = jvp_base();
      a.v = w.p; a.out = w.v; a.ndots = 1; a.dw[0] = w.p; a.sums = ctx->bctl->sums;
      a.active = &ctx->bctl->active;
      if (fd_norms) a.vn2 = vv.pn2;
      jfnk_status s = jvp(a, it);
      if (s) return s;
      int e2 = tm_begin(ctx, KC_BICG, nv * (4 * s_ + 2 * ss()), it);
      e = launch_cg(2, ts, tj, td, N, vv, ctx->bctl, ctx->red, it, o.tol_krylov, ctx->stream);
      tm_end(ctx, e2);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cg update");
      CK(cudaEventRecord(ctx->iter_ev[it % (kLookahead + 1)], ctx->stream), "event record");
    }
    jfnk_status s = sync_read(ctx->bctl, sizeof(BicgCtl));
    if (s) return s;
    BicgCtl c;
    std::memcpy(&c, ctx->hbuf, sizeof(BicgCtl));
    tm_harvest(ctx, c.its, -1.0);
    rep.krylov_its += c.its;
    rep.jvp_calls += c.its;
    if (c.nonfinite) *kstatus = JFNK_E_NONFINITE;
    else if (c.breakdown) *kstatus = JFNK_E_BREAKDOWN;
    else if (!c.converged) *kstatus = JFNK_E_NOT_CONVERGED;
    return JFNK_OK;
  }

  // ---- one nonlinear solve F(x; b) = 0 from the current x ---------------
  // denom > 0 overrides ||F(x0)|| as the Eq. 5 denominator.
  jfnk_status newton(int* nstatus, double denom, bool linear_once) {
    jfnk_ctx::Ws& w = ctx->ws;
    const void* bb = P.bvp ? nullptr : w.b;
    jfnk_status s = residual(x, nullptr, 0.0, F, nullptr, tj != ts ? x32 : nullptr, sc, ts, bb);
    if (s) return s;
    s = sync_read(sc, 16);
    if (s) return s;
    double fnorm = std::sqrt(ctx->hbuf[0]);
    const double f0 = denom > 0 ? denom : fnorm;
    rep.res0 = f0;
    for (double& a : rep.ls_alpha) a = 0.0;
    int nits = 0;   // Newton iterations of this solve
    *nstatus = JFNK_OK;
    for (int k = 0; k <= o.max_newton; ++k) {
      if (!std::isfinite(fnorm)) { *nstatus = JFNK_E_NONFINITE; break; }
      if (f0 == 0.0 || fnorm / f0 < o.tol_newton) { *nstatus = JFNK_OK; break; }
      if (k == o.max_newton || (linear_once && k == 1)) { *nstatus = JFNK_E_NOT_CONVERGED; break; }
      if (o.lin == 1 && tj != ts) {
        // FD needs F at the linearisation point in the JVP precision
        s = residual(x32, nullptr, 0.0, w.F32, nullptr, nullptr, nullptr, tj, P.bvp ? nullptr : w.b32);
        if (s) return s;
      }
      int kst = 0;
      s = (o.krylov == JFNK_BICGSTAB) ? bicgstab(&kst) : (o.krylov == JFNK_CG ? cg(&kst) : gmres_auto(&kst));
      if (s) return s;
      s = precond_solution();
      if (s) return s;
      if (kst == JFNK_E_BREAKDOWN || kst == JFNK_E_NONFINITE) { *nstatus = kst; break; }
      if (kst == JFNK_E_NOT_CONVERGED) rep.krylov_failures += 1;
      // backtracking line search on ||F||, decided on the device (LsCtl): every trial
      // alpha = 1, 1/2, ..., down to the smallest is queued at once, the last block of
      // each trial takes the Armijo decision, and the trials after the accepted one do
      // nothing, so Ft, xt and st hold the accepted state. One read-back per Newton
      // step. The linear Born solve takes the full step.
      int ntrial = 1;
      if (!linear_once)
        for (double a = 1.0; a * 0.5 >= o.ls_min_alpha; a *= 0.5) ++ntrial;
      cudaError_t e = launch_ls_begin(ctx->lsc, fnorm, o.ls_c1, o.ls_min_alpha, linear_once ? 1 : 0, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "line search");
      for (int q = 0; q < ntrial; ++q) {
        s = residual(x, w.d, 1.0, Ft, xt, tj != ts ? x32t : nullptr, st, ts, bb, ctx->lsc, q);
        if (s) return s;
      }
      CK(cudaMemcpyAsync((char*)ctx->hbuf + 4096, ctx->lsc, sizeof(LsCtl), cudaMemcpyDeviceToHost, ctx->stream),
         "read-back");
      s = sync_read(st, 16);
      if (s) return s;
      LsCtl ls;
      std::memcpy(&ls, (char*)ctx->hbuf + 4096, sizeof(LsCtl));
      tm_harvest(ctx, ls.backtracks + 1, -1.0);
      if (!ls.done) return fail(ctx, JFNK_E_CUDA, "line search: no trial was accepted");
      const double ft = ls.ft;
      rep.ls_backtracks += ls.backtracks;
      rep.ls_failures += ls.failures;
      if (nits < 16) rep.ls_alpha[nits] = ls.alpha_acc;
      ++nits;
      std::swap(x, xt); std::swap(F, Ft); std::swap(sc, st); std::swap(x32, x32t);
      fnorm = ft;
      rep.newton_its += 1;
    }
    rep.res_final = fnorm;
    return JFNK_OK;
  }
};

}  // namespace

namespace jfnk {
size_t workspace_estimate(const jfnk_problem* pr, const jfnk_opts* o) {
  int ts, tj, tb;
  if (!pr || !o || !prec_types(o->prec, &ts, &tj, &tb) || pr->nx < 1 || pr->ny < 1) return 0;
  const size_t nf = (size_t)pde_nfields(pr->pde);
  const size_t N = (size_t)pr->nx * pr->ny * nf;
  const size_t ss = vt_size(ts), sj = vt_size(tj), sb = vt_size(tb);
  size_t b = N * (7 * ss + 8 + 3 * sj) + (tj != ts ? 4 * N * sj : 0);
  const size_t m = o->restart > 0 ? (size_t)o->restart : (size_t)kTuneMaxRestart;
  b += (o->krylov == JFNK_GMRES) ? (m + 1) * N * sb + N * ss : 6 * N * sj;
  if (o->krylov == JFNK_GMRES && tj == VT_F32 && tb == VT_F32) b += 3 * N * sj;   // fused Arnoldi buffers
  b += (size_t)2048 * kMaxK * 8 + 65536;   // reductions and control blocks
  if (pr->pde == JFNK_MAXWELL_TE2D) b += (size_t)pr->nx * pr->ny * 3 * 12;
  if (pr->pde == JFNK_MAXWELL_VEC2D) b += (size_t)pr->nx * pr->ny * 4 * 12;
  return b;
}
}  // namespace jfnk

// ============================================================================
// C ABI
// ============================================================================
static jfnk_status jfnk_create_impl(jfnk_ctx* ctx, int device, size_t hbm_budget, void* cuda_stream) {
  ctx->device = device;
  ctx->budget = hbm_budget;
  CK(cudaSetDevice(device), "cudaSetDevice");
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "stream create");
    ctx->own_stream = true;
  }
  jfnk_status s;
  if ((s = dalloc(ctx, (void**)&ctx->dsc, 64 * sizeof(double), nullptr)) ||
      (s = dalloc(ctx, (void**)&ctx->gctl, sizeof(GmresCtl), nullptr)) ||
      (s = dalloc(ctx, (void**)&ctx->bctl, sizeof(BicgCtl), nullptr)) ||
      (s = dalloc(ctx, (void**)&ctx->lsc, sizeof(LsCtl), nullptr)) ||
      (s = dalloc(ctx, (void**)&ctx->red.counter, 256, nullptr)) ||
      (s = dalloc(ctx, (void**)&ctx->derr, 256, nullptr)))
    return s;
  CK(cudaMemset(ctx->derr, 0, 256), "memset");
  CK(cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device), "device attribute");
  ctx->stream_ok = true;
  CK(cudaMemset(ctx->dsc, 0, 64 * sizeof(double)), "memset");
  CK(cudaMemset(ctx->gctl, 0, sizeof(GmresCtl)), "memset");
  CK(cudaMemset(ctx->bctl, 0, sizeof(BicgCtl)), "memset");
  CK(cudaMemset(ctx->red.counter, 0, 256), "memset");
  int* hf = nullptr;
  CK(cudaHostAlloc((void**)&hf, 64, cudaHostAllocMapped), "cudaHostAlloc");
  ctx->hflag = hf;
  CK(cudaHostGetDevicePointer((void**)&ctx->hflag_dev, hf, 0), "cudaHostGetDevicePointer");
  CK(cudaHostAlloc((void**)&ctx->hbuf, 16384, cudaHostAllocDefault), "cudaHostAlloc");
  volatile int* dflag = (volatile int*)ctx->hflag_dev;
  CK(cudaMemcpy((char*)ctx->gctl + offsetof(GmresCtl, host_active), &dflag, sizeof(dflag), cudaMemcpyHostToDevice),
     "ctl init");
  CK(cudaMemcpy((char*)ctx->bctl + offsetof(BicgCtl, host_active), &dflag, sizeof(dflag), cudaMemcpyHostToDevice),
     "ctl init");
  for (int q = 0; q <= kLookahead; ++q)
    CK(cudaEventCreateWithFlags(&ctx->iter_ev[q], cudaEventDisableTiming), "event create");
  return JFNK_OK;
}

extern "C" {

const char* jfnk_status_string(int s) {
  switch (s) {
    case JFNK_OK: return "ok";
    case JFNK_E_INVALID: return "invalid argument";
    case JFNK_E_OOM: return "out of memory budget";
    case JFNK_E_CUDA: return "CUDA error";
    case JFNK_E_NOT_CONVERGED: return "not converged";
    case JFNK_E_BREAKDOWN: return "Krylov breakdown";
    case JFNK_E_NONFINITE: return "non-finite value";
    case JFNK_E_LINESEARCH: return "line search failure";
    case JFNK_E_TIMEOUT: return "timeout";
    case JFNK_E_BUSY: return "busy";
  }
  return "unknown status";
}

void jfnk_default_opts(jfnk_opts* o, int prec) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  const bool lowp = (prec == JFNK_FP32);
  o->lin = JFNK_AD;
  o->krylov = JFNK_GMRES;
  o->prec = prec;
  o->restart = 30;
  o->max_newton = 15;
  o->max_krylov = 100;
  o->tol_newton = lowp ? 1e-4 : 1e-6;
  o->tol_krylov = lowp ? 1e-6 : 1e-8;
  o->fd_rule = JFNK_EPS_SCALED;
  o->fd_eps = 0.0;
  o->ls_c1 = 1e-4;
  o->ls_min_alpha = 1.0 / 1024.0;
  o->born_start = 1;
  o->ortho = JFNK_CGS2;
  o->precond = JFNK_PRECOND_NONE;
  o->precond_damping = 0.5;
}

jfnk_status jfnk_create(jfnk_ctx** out, int device, size_t hbm_budget, void* cuda_stream) {
  if (!out) return JFNK_E_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return JFNK_E_INVALID;
  }
  jfnk_ctx* ctx = new jfnk_ctx();
  jfnk_status st = jfnk_create_impl(ctx, device, hbm_budget, cuda_stream);
  if (st != JFNK_OK) {
    jfnk_destroy(ctx);
    return st;
  }
  *out = ctx;
  return JFNK_OK;
}

void jfnk_destroy(jfnk_ctx* ctx) {
  if (!ctx) return;
  if (ctx->server) { delete ctx->server; ctx->server = nullptr; }
  if (ctx->batch) { delete ctx->batch; ctx->batch = nullptr; }
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ws_free(ctx);
  cudaFree(ctx->eps64); cudaFree(ctx->eps32); cudaFree(ctx->src64); cudaFree(ctx->src32);
  cudaFree(ctx->dsc); cudaFree(ctx->gctl); cudaFree(ctx->bctl); cudaFree(ctx->lsc);
  cudaFree(ctx->red.partials); cudaFree(ctx->red.counter); cudaFree(ctx->jscratch); cudaFree(ctx->derr);
  if (ctx->hflag) cudaFreeHost((void*)ctx->hflag);
  if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
  for (int q = 0; q <= kLookahead; ++q) if (ctx->iter_ev[q]) cudaEventDestroy(ctx->iter_ev[q]);
  for (cudaEvent_t e : ctx->tm.pool) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaGetLastError();
  delete ctx;
}

const char* jfnk_last_error(const jfnk_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

jfnk_status jfnk_set_problem(jfnk_ctx* ctx, const jfnk_problem* pr) {
  if (!ctx || !pr) return JFNK_E_INVALID;
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  ProbDev P;
  std::string why;
  if (!make_probdev(pr, &P, &why)) return fail(ctx, JFNK_E_INVALID, why);
  const int pde = pr->pde;
  cudaStreamSynchronize(ctx->stream);
  // problem-owned arrays
  cudaFree(ctx->eps64); cudaFree(ctx->eps32); cudaFree(ctx->src64); cudaFree(ctx->src32);
  ctx->eps64 = nullptr; ctx->eps32 = nullptr; ctx->src64 = nullptr; ctx->src32 = nullptr;
  const long long n = P.ncell;
  if (pde == JFNK_MAXWELL_TE2D || pde == JFNK_MAXWELL_VEC2D) {
    const double* hin[2] = {pr->aux[0], pr->aux[1]};
    const long long cnt[2] = {n, pde_source_planes(pde) * n};
    double** d64[2] = {&ctx->eps64, &ctx->src64};
    float** d32[2] = {&ctx->eps32, &ctx->src32};
    for (int q = 0; q < 2; ++q) {
      if (!hin[q]) continue;
      CK(cudaMalloc((void**)d64[q], cnt[q] * 8), "cudaMalloc aux");
      CK(cudaMalloc((void**)d32[q], cnt[q] * 4), "cudaMalloc aux");
      CK(cudaMemcpy(*d64[q], hin[q], cnt[q] * 8, cudaMemcpyDefault), "copy aux");
      cudaError_t e = launch_cast(VT_F64, VT_F32, cnt[q], *d64[q], *d32[q], 1.0, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cast aux");
    }
    CK(cudaStreamSynchronize(ctx->stream), "aux");
  }
  P.eps64 = ctx->eps64; P.eps32 = ctx->eps32; P.src64 = ctx->src64; P.src32 = ctx->src32;
  ctx->P = P;
  ctx->prob = *pr;
  ctx->N = P.ncell * P.nf;
  ctx->have_prob = true;
  if (ctx->ws.ok && ctx->ws.N != ctx->N) ws_free(ctx);
  return ensure_red(ctx);
}

jfnk_status jfnk_residual(jfnk_ctx* ctx, int prec, const void* x, const void* b, void* F) {
  if (!ctx || !x || !F) return JFNK_E_INVALID;
  if (!ctx->have_prob) return fail(ctx, JFNK_E_INVALID, "no problem set");
  if (prec != JFNK_FP64 && prec != JFNK_FP32) return fail(ctx, JFNK_E_INVALID, "prec must be FP64 or FP32");
  if (ctx->P.cfl > 0.0)
    return fail(ctx, JFNK_E_INVALID, "adaptive time step (Courant number > 0): the step exists only inside "
                                     "jfnk_solve; install the problem with C = 0 and dt");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaError_t e = launch_residual(ctx->P, prec == JFNK_FP64 ? VT_F64 : VT_F32, x, nullptr, 0.0,
                                  ctx->P.bvp ? nullptr : b, F, nullptr, nullptr, ctx->red, nullptr, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "residual kernel");
  return JFNK_OK;
}

jfnk_status jfnk_jvp(jfnk_ctx* ctx, int lin, int prec, const void* x, const void* v, const void* b, void* F_out,
                     void* Jv_out, double fd_eps) {
  if (!ctx || !x || !v || !Jv_out) return JFNK_E_INVALID;
  if (!ctx->have_prob) return fail(ctx, JFNK_E_INVALID, "no problem set");
  if (lin != JFNK_AD && lin != JFNK_FD) return fail(ctx, JFNK_E_INVALID, "lin must be AD or FD");
  if (prec != JFNK_FP64 && prec != JFNK_FP32) return fail(ctx, JFNK_E_INVALID, "prec must be FP64 or FP32");
  if (ctx->P.cfl > 0.0)
    return fail(ctx, JFNK_E_INVALID, "adaptive time step (Courant number > 0): the step exists only inside "
                                     "jfnk_solve; install the problem with C = 0 and dt");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const int t = prec == JFNK_FP64 ? VT_F64 : VT_F32;
  const long long N = ctx->N;
  if (ctx->P.bvp) b = nullptr;
  JvpArgs a;
  std::memset(&a, 0, sizeof(a));
  a.lin = lin; a.t = t; a.tv = t; a.x = x; a.v = v; a.b = b; a.out = Jv_out; a.c_jv = 1.0;
  a.err = ctx->derr;
  if (lin == JFNK_AD) {
    a.F = F_out;
  } else {
    void* Fx = F_out;
    if (!Fx) {
      const size_t need = (size_t)N * 8;
      if (ctx->jscratch_bytes < need) {
        cudaStreamSynchronize(ctx->stream);
        if (ctx->jscratch) { cudaFree(ctx->jscratch); ctx->allocated -= ctx->jscratch_bytes; }
        ctx->jscratch = nullptr;
        ctx->jscratch_bytes = 0;
        jfnk_status s = dalloc(ctx, &ctx->jscratch, need, nullptr);
        if (s) return s;
        ctx->jscratch_bytes = need;
      }
      Fx = ctx->jscratch;
    }
    cudaError_t e = launch_residual(ctx->P, t, x, nullptr, 0.0, b, Fx, nullptr, nullptr, ctx->red, nullptr,
                                    ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "residual kernel");
    a.Fx = Fx;
    a.eps_fixed = fd_eps;
    a.eps_rule = JFNK_EPS_SCALED;
    if (fd_eps <= 0.0) {
      const void* aa[3] = {x, v, nullptr};
      const void* bb[3] = {nullptr, nullptr, nullptr};
      e = launch_vdots(t, N, 2, aa, bb, ctx->dsc + 4, ctx->red, nullptr, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "norm kernel");
      a.xn2 = ctx->dsc + 4;
      a.vn2 = ctx->dsc + 5;
    }
  }
  cudaError_t e = launch_jvp(ctx->P, a, ctx->red, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "jvp kernel");
  return JFNK_OK;
}

static jfnk_status validate_opts(jfnk_ctx* ctx, const jfnk_opts* o) {
  int ts, tj, tb;
  if (!prec_types(o->prec, &ts, &tj, &tb)) return fail(ctx, JFNK_E_INVALID, "bad precision");
  if (o->lin != JFNK_AD && o->lin != JFNK_FD) return fail(ctx, JFNK_E_INVALID, "bad linearisation");
  if (o->krylov != JFNK_GMRES && o->krylov != JFNK_BICGSTAB && o->krylov != JFNK_CG)
    return fail(ctx, JFNK_E_INVALID, "krylov must be GMRES, BiCGSTAB or CG");
  if (o->krylov == JFNK_GMRES && (o->restart < 0 || o->restart > JFNK_MAX_RESTART))
    return fail(ctx, JFNK_E_INVALID, "restart out of range (0: tuned)");
  if (o->krylov != JFNK_GMRES && o->prec == JFNK_MIXED_BF16)
    return fail(ctx, JFNK_E_INVALID, "BF16 storage applies to the GMRES basis only");
  if (o->max_newton < 0 || o->max_krylov < 1) return fail(ctx, JFNK_E_INVALID, "bad iteration limits");
  if (!(o->tol_newton >= 0) || !(o->tol_krylov >= 0)) return fail(ctx, JFNK_E_INVALID, "bad tolerances");
  if (!(o->ls_min_alpha > 0.0 && o->ls_min_alpha <= 1.0)) return fail(ctx, JFNK_E_INVALID, "bad ls_min_alpha");
  if (o->fd_rule != JFNK_EPS_SCALED && o->fd_rule != JFNK_EPS_PAPER) return fail(ctx, JFNK_E_INVALID, "bad fd_rule");
  if (o->ortho != JFNK_CGS2 && o->ortho != JFNK_DCGS2 && o->ortho != JFNK_DCGS2_FUSED)
    return fail(ctx, JFNK_E_INVALID, "bad ortho");
  if (o->precond != JFNK_PRECOND_NONE && o->precond != JFNK_PRECOND_CSLP)
    return fail(ctx, JFNK_E_INVALID, "bad precond");
  if (o->precond == JFNK_PRECOND_CSLP) {
    if (ctx->P.pde != JFNK_MAXWELL_VEC2D)
      return fail(ctx, JFNK_E_INVALID, "the CSLP preconditioner belongs to the vector Maxwell problem");
    if (o->krylov != JFNK_GMRES || o->prec == JFNK_MIXED_BF16 || o->ortho == JFNK_DCGS2_FUSED)
      return fail(ctx, JFNK_E_INVALID, "the CSLP preconditioner needs GMRES with a CGS2 or delayed-CGS2 FP64/FP32 basis");
    if (!(o->precond_damping >= 0.0 && std::isfinite(o->precond_damping)))
      return fail(ctx, JFNK_E_INVALID, "bad precond_damping");
  }
  if (o->krylov == JFNK_GMRES && o->ortho != JFNK_CGS2 && !(ctx->stream_ok && stream_supported(ctx->N)))
    return fail(ctx, JFNK_E_INVALID, "delayed CGS2 needs the bulk-copy streaming kernels (unknowns a multiple of 8, "
                                     "JFNK_TUNE_BULK_COPY on)");
  if (o->krylov == JFNK_GMRES && o->ortho == JFNK_DCGS2_FUSED) {
    const bool ok = o->lin == JFNK_AD && tb == VT_F32 && tj == VT_F32 && ctx->stream_ok &&
                    dcgs_fused_supported(ctx->P, o->restart > 0 ? o->restart : kTuneMaxRestart, ctx->nsm);
    if (!ok)
      return fail(ctx, JFNK_E_INVALID, "the one-pass delayed CGS2 form needs the AD JVP, FP32 JVP and basis, and a "
                                       "2D problem with face neighbours only whose rows fit its shared-memory plan");
  }
  return JFNK_OK;
}

jfnk_status jfnk_solve(jfnk_ctx* ctx, const jfnk_opts* opts, const double* x_prev, double* x_inout, int steps,
                       jfnk_report* rep) {
  if (!ctx || !opts || !x_inout) return JFNK_E_INVALID;
  if (!ctx->have_prob) return fail(ctx, JFNK_E_INVALID, "no problem set");
  jfnk_status s = validate_opts(ctx, opts);
  if (s) return s;
  if (!ctx->P.bvp && steps < 1) return fail(ctx, JFNK_E_INVALID, "steps must be >= 1");
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  s = ensure_ws(ctx, opts->prec, opts->restart > 0 ? opts->restart : kTuneMaxRestart, opts->krylov);
  if (s) return s;
  s = ensure_red(ctx);
  if (s) return s;
  Solver sv;
  sv.ctx = ctx;
  sv.o = *opts;
  prec_types(opts->prec, &sv.ts, &sv.tj, &sv.tb);
  sv.td = sv.ts;
  sv.N = ctx->N;
  sv.P = ctx->P;
  std::memset(&sv.rep, 0, sizeof(sv.rep));
  jfnk_ctx::Ws& w = ctx->ws;
  sv.x = w.x; sv.xt = w.xt; sv.F = w.F; sv.Ft = w.Ft; sv.x32 = w.x32; sv.x32t = w.x32t;
  sv.sc = ctx->dsc + 0; sv.st = ctx->dsc + 2;
  const long long N = ctx->N;
  const size_t bytes64 = (size_t)N * 8;
  // initial state into the FP64 staging buffer, then into the state precision
  const double* src = x_prev ? x_prev : x_inout;
  CK(cudaMemcpyAsync(w.user, src, bytes64, cudaMemcpyDefault, ctx->stream), "copy in");
  if (sv.ts == VT_F64) {
    CK(cudaMemcpyAsync(sv.x, w.user, bytes64, cudaMemcpyDeviceToDevice, ctx->stream), "copy in");
  } else {
    s = sv.cast(VT_F64, VT_F32, w.user, sv.x, 1.0);
    if (s) return s;
  }
  jfnk_status first_bad = JFNK_OK;
  const size_t sbytes = (size_t)N * vt_size(sv.ts);
  if (ctx->P.bvp) {
    double denom = 0.0;
    if (opts->born_start && (ctx->P.pde == JFNK_MAXWELL_TE2D || ctx->P.pde == JFNK_MAXWELL_VEC2D)) {
      // Born start: the chi3 = 0 problem solved once from zero
      Solver lin = sv;
      lin.P.p1 = 0.0;
      CK(cudaMemsetAsync(lin.x, 0, sbytes, ctx->stream), "memset");
      if (lin.x32) CK(cudaMemsetAsync(lin.x32, 0, (size_t)N * 4, ctx->stream), "memset");
      int ns = 0;
      s = lin.newton(&ns, 0.0, true);
      if (s) return s;
      sv.x = lin.x; sv.xt = lin.xt; sv.F = lin.F; sv.Ft = lin.Ft; sv.x32 = lin.x32; sv.x32t = lin.x32t;
      sv.sc = lin.sc; sv.st = lin.st;
      sv.rep.krylov_its += lin.rep.krylov_its;
      sv.rep.jvp_calls += lin.rep.jvp_calls;
    }
    int ns = 0;
    s = sv.newton(&ns, denom, false);
    if (s) return s;
    sv.rep.steps_done = 1;
    sv.rep.status = ns;
    if (ns != JFNK_OK) first_bad = (jfnk_status)ns;
    if (!(sv.rep.res0 == 0.0 || sv.rep.res_final / sv.rep.res0 < 100.0 * opts->tol_newton)) sv.rep.steps_failed = 1;
  } else {
    for (int step = 0; step < steps; ++step) {
      sv.rep.dt_last = ctx->prob.dt;
      if (sv.P.cfl > 0.0) {
        double dt = 0.0;
        s = sv.cfl_step(&dt);
        if (s) return s;
        sv.rep.dt_last = dt;
        if (!std::isfinite(dt)) {
          sv.rep.status = JFNK_E_NONFINITE;
          sv.rep.steps_failed += 1;
          if (first_bad == JFNK_OK) first_bad = JFNK_E_NONFINITE;
          break;
        }
      }
      // x^n -> b_n; x starts from x^n
      const int evr = tm_begin(ctx, KC_RHS, (double)N * 2 * vt_size(sv.ts), -1);
      cudaError_t e = launch_rhs(sv.P, sv.ts, sv.x, w.b, ctx->stream);
      tm_end(ctx, evr);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "rhs kernel");
      if (sv.tj != sv.ts) {
        s = sv.cast(sv.ts, sv.tj, w.b, w.b32, 1.0);
        if (s) return s;
      }
      int ns = 0;
      s = sv.newton(&ns, 0.0, false);
      if (s) return s;
      sv.rep.steps_done += 1;
      sv.rep.status = ns;
      if (!(sv.rep.res0 == 0.0 || sv.rep.res_final / sv.rep.res0 < 100.0 * opts->tol_newton))
        sv.rep.steps_failed += 1;
      if (ns != JFNK_OK && first_bad == JFNK_OK) first_bad = (jfnk_status)ns;
      if (ns == JFNK_E_NONFINITE || ns == JFNK_E_BREAKDOWN) break;
    }
  }
  // result back to the caller's FP64 array
  if (sv.ts == VT_F64) {
    CK(cudaMemcpyAsync(x_inout, sv.x, bytes64, cudaMemcpyDefault, ctx->stream), "copy out");
  } else {
    s = sv.cast(VT_F32, VT_F64, sv.x, w.user, 1.0);
    if (s) return s;
    CK(cudaMemcpyAsync(x_inout, w.user, bytes64, cudaMemcpyDefault, ctx->stream), "copy out");
  }
  CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  tm_harvest(ctx, 0, -1.0);
  // keep the workspace buffers consistent with the swapped pointers
  w.x = sv.x; w.xt = sv.xt; w.F = sv.F; w.Ft = sv.Ft; w.x32 = sv.x32; w.x32t = sv.x32t;
  sv.rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = sv.rep;
  return first_bad;
}

jfnk_status jfnk_set_timing(jfnk_ctx* ctx, int enable) {
  if (!ctx) return JFNK_E_INVALID;
  ctx->tm.on = enable != 0;
  return JFNK_OK;
}

int jfnk_kernel_stats(jfnk_ctx* ctx, const char** names, long long* launches, double* total_ms, double* bytes,
                      int cap) {
  if (!ctx) return 0;
  int n = 0;
  for (int c = 0; c < KC_COUNT && n < cap; ++c, ++n) {
    if (names) names[n] = kKClassNames[c];
    if (launches) launches[n] = ctx->tm.launches[c];
    if (total_ms) total_ms[n] = ctx->tm.ms[c];
    if (bytes) bytes[n] = ctx->tm.bytes[c];
  }
  if (n < cap) {   // every launch, including those a converged Krylov loop turned into no-ops
    if (names) names[n] = "all_launches";
    if (launches) launches[n] = ctx->tm.total_launches;
    if (total_ms) total_ms[n] = 0.0;
    if (bytes) bytes[n] = 0.0;
    ++n;
  }
  return n;
}

void jfnk_reset_stats(jfnk_ctx* ctx) {
  if (!ctx) return;
  for (int c = 0; c < KC_COUNT; ++c) { ctx->tm.launches[c] = 0; ctx->tm.ms[c] = 0; ctx->tm.bytes[c] = 0; }
  ctx->tm.total_launches = 0;
}

jfnk_status jfnk_submit(jfnk_ctx* ctx, const jfnk_problem* prob, const jfnk_opts* opts, const double* x0,
                        double* x_out, int steps, unsigned long long* ticket) {
  if (!ctx || !prob || !opts || !x0 || !x_out || !ticket) return JFNK_E_INVALID;
  // one single-solve worker beside the batch engine: a large solve fills the GPU by itself, and four
  // concurrent large solves next to the batch engine's multi-branch graph replays faulted the device
  // intermittently (an unexplained illegal access) where one at a time never did
  if (!ctx->server) ctx->server = new jfnk::Server(ctx->device, ctx->budget, kServeSlotWorkers);
  return ctx->server->submit(prob, opts, x0, x_out, steps, ticket);
}

jfnk_status jfnk_solve_batch(jfnk_ctx* ctx, int count, const jfnk_problem* probs, const jfnk_opts* opts,
                             const double* const* x_prev, double* const* x_inout, const int* steps,
                             jfnk_report* reps, int* statuses) {
  if (!ctx || count < 0) return JFNK_E_INVALID;
  if (count == 0) return JFNK_OK;
  if (!probs || !opts || !x_inout || !steps) return fail(ctx, JFNK_E_INVALID, "null array");
  size_t need = 0;
  for (int i = 0; i < count; ++i) {
    std::string why;
    if (!jfnk::BatchEngine::supports(&probs[i], &opts[i], &why))
      return fail(ctx, JFNK_E_INVALID, "problem " + std::to_string(i) + ": " + why);
    if (!x_inout[i]) return fail(ctx, JFNK_E_INVALID, "problem " + std::to_string(i) + ": null state");
    if (probs[i].pde != JFNK_MAXWELL_TE2D && steps[i] < 1)
      return fail(ctx, JFNK_E_INVALID, "problem " + std::to_string(i) + ": steps must be >= 1");
    need += jfnk::BatchEngine::workspace_bytes(&probs[i], &opts[i]);
  }
  if (ctx->budget && ctx->allocated + need > ctx->budget)
    return fail(ctx, JFNK_E_OOM, "batch workspace of " + std::to_string(need) + " bytes exceeds the HBM budget");
  CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");   // caller's inputs are ready
  if (!ctx->batch) {
    ctx->batch = new jfnk::BatchEngine(ctx->device);
    ctx->batch->set_tile_override(ctx->batch_tile);
  }
  jfnk::BatchEngine& E = *ctx->batch;
  std::string why;
  for (int i = 0; i < count; ++i) {
    jfnk::BatRequest r;
    r.prob = probs[i];
    r.opts = opts[i];
    r.x0 = (x_prev && x_prev[i]) ? x_prev[i] : x_inout[i];
    r.x_out = x_inout[i];
    r.steps = steps[i];
    r.tag = (unsigned long long)i;
    jfnk_status s = E.admit(r, &why);
    if (s) {
      E.drop_all();
      return fail(ctx, s, "admit " + std::to_string(i) + ": " + why);
    }
  }
  // every solve ends after a bounded number of phases: stop replaying past that bound
  long long bound = 0;
  for (int i = 0; i < count; ++i) {
    const jfnk_opts& o = opts[i];
    const long long per_newton = (long long)o.max_krylov * (4LL * o.restart + 3) + 16;
    const long long solves = (probs[i].pde == JFNK_MAXWELL_TE2D) ? 2 : steps[i];
    bound = std::max(bound, solves * (o.max_newton + 1) * per_newton + 8);
  }
  std::vector<jfnk_status> st(count, JFNK_OK);
  std::vector<jfnk::BatResult> fin;
  long long phases = 0;
  while (E.active() > 0) {
    if (phases > bound) {
      E.drop_all();
      return fail(ctx, JFNK_E_TIMEOUT, "batch: a solve did not finish within its phase bound");
    }
    phases += E.launches_per_replay();
    fin.clear();
    jfnk_status s = E.advance(&fin, &why);
    if (s) {
      E.drop_all();
      return fail(ctx, s, "batch: " + why);
    }
    for (const jfnk::BatResult& r : fin) {
      st[r.tag] = r.status;
      if (reps) reps[r.tag] = r.rep;
    }
  }
  jfnk_status first = JFNK_OK;
  for (int i = 0; i < count; ++i) {
    if (statuses) statuses[i] = st[i];
    if (first == JFNK_OK && st[i] != JFNK_OK) first = st[i];
  }
  return first;
}

jfnk_status jfnk_tune(jfnk_ctx* ctx, int knob, long long value) {
  if (!ctx) return JFNK_E_INVALID;
  switch (knob) {
    case JFNK_TUNE_BATCH_TILE: {
      if (value < 0) return fail(ctx, JFNK_E_INVALID, "batch tile: cells must be >= 0");
      const int t = value == 0 ? 0 : (int)std::max<long long>(256, std::min<long long>(2048, value / 256 * 256));
      ctx->batch_tile = t;
      if (ctx->batch) ctx->batch->set_tile_override(t);
      return JFNK_OK;
    }
    case JFNK_TUNE_BULK_COPY:
      if (value != 0 && value != 1) return fail(ctx, JFNK_E_INVALID, "bulk copy: 0 or 1");
      ctx->stream_ok = value == 1;
      return JFNK_OK;
    default:
      return fail(ctx, JFNK_E_INVALID, "unknown tuning knob");
  }
}

jfnk_status jfnk_batch_stats(jfnk_ctx* ctx, long long* kernel_launches, int* tile_cells, int pde, int prec,
                             int nx, int ny) {
  if (!ctx) return JFNK_E_INVALID;
  if (kernel_launches) *kernel_launches = ctx->batch ? ctx->batch->kernel_launches() : 0;
  if (tile_cells) {
    *tile_cells = 0;
    if (ctx->batch) *tile_cells = ctx->batch->tuned_tile(pde, prec, (long long)nx * ny);
  }
  return JFNK_OK;
}

jfnk_status jfnk_poll(jfnk_ctx* ctx, unsigned long long ticket, jfnk_report* rep) {
  if (!ctx) return JFNK_E_INVALID;
  if (!ctx->server) return fail(ctx, JFNK_E_INVALID, "unknown ticket");
  return ctx->server->poll(ticket, rep);
}

}  // extern "C"
