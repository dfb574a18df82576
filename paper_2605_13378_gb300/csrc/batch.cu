// batch.cu -- host side of the batched solver (see batch_engine.h): slot
// workspaces, the (solve, tile) work lists per (PDE, precision) group, the
// captured graph of batch-kernel launches, and the tile-size autotuner.
#include "batch_engine.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "krylov.h"

namespace jfnk {

cudaError_t batch_launch(int pde, int ts, int tj, const BatLaunch& L, int grid, cudaStream_t st) {
  switch (pde) {
    case JFNK_BURGERS1D: return batch_launch_burgers(ts, tj, L, grid, st);
    case JFNK_ALLEN_CAHN2D: return batch_launch_allen_cahn(ts, tj, L, grid, st);
    case JFNK_SU_OLSON2D: return batch_launch_su_olson(ts, tj, L, grid, st);
    case JFNK_MAXWELL_TE2D: return batch_launch_maxwell(ts, tj, L, grid, st);
    case JFNK_BURGERS2D: return batch_launch_burgers2d(ts, tj, L, grid, st);
  }
  return cudaErrorInvalidValue;
}

int batch_grid_cap(int pde, int ts, int tj, int nsm) {
  int occ = 1;
  switch (pde) {
    case JFNK_BURGERS1D: occ = batch_occ_burgers(ts, tj); break;
    case JFNK_ALLEN_CAHN2D: occ = batch_occ_allen_cahn(ts, tj); break;
    case JFNK_SU_OLSON2D: occ = batch_occ_su_olson(ts, tj); break;
    case JFNK_MAXWELL_TE2D: occ = batch_occ_maxwell(ts, tj); break;
    case JFNK_BURGERS2D: occ = batch_occ_burgers2d(ts, tj); break;
  }
  return std::max(1, occ) * nsm;
}

namespace {

constexpr int kTileCands[] = {256, 512, 1024, 2048};

int pair_of(int prec, int* ts, int* tj) {
  switch (prec) {
    case JFNK_FP64: *ts = VT_F64; *tj = VT_F64; return 0;
    case JFNK_FP32: *ts = VT_F32; *tj = VT_F32; return 1;
    case JFNK_MIXED_FP32: *ts = VT_F64; *tj = VT_F32; return 2;
  }
  return -1;
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte layout of one slot. With `base` null only the total is computed.
size_t carve(const jfnk_problem* pr, const jfnk_opts* o, unsigned char* base, BatDesc* D) {
  int ts = 0, tj = 0;
  pair_of(o->prec, &ts, &tj);
  const long long ncell = (long long)pr->nx * pr->ny;
  const int nf = pde_nfields(pr->pde);
  const size_t N = (size_t)ncell * nf;
  const size_t ss = vt_size(ts), sj = vt_size(tj);
  const bool mixed = ts != tj;
  const size_t nunit = (size_t)((ncell + kBatUnit - 1) / kBatUnit);
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = base ? (void*)(base + off) : nullptr;
    off += al256(bytes);
    return p;
  };
  void* st = take(sizeof(BatState));
  void* io = take(N * 8);
  void* x0 = take(N * ss);
  void* x1 = take(N * ss);
  void* F0 = take(N * ss);
  void* F1 = take(N * ss);
  void* b = take(N * ss);
  void* d = take(N * ss);
  void* x320 = mixed ? take(N * 4) : nullptr;
  void* x321 = mixed ? take(N * 4) : nullptr;
  void* b32 = mixed ? take(N * 4) : nullptr;
  void* F32 = (mixed && o->lin == JFNK_FD) ? take(N * 4) : nullptr;
  void* rhs = take(N * sj);
  void* w = take(N * sj);
  void* V = take((size_t)(o->restart + 1) * N * sj);
  void* part = take(nunit * kBatPart * 8);
  void* e64 = nullptr; void* s64 = nullptr; void* e32 = nullptr; void* s32 = nullptr;
  if (pr->pde == JFNK_MAXWELL_TE2D) {
    if (pr->aux[0]) { e64 = take(ncell * 8); e32 = take(ncell * 4); }
    if (pr->aux[1]) { s64 = take(2 * ncell * 8); s32 = take(2 * ncell * 4); }
  }
  if (D) {
    D->st = (BatState*)st;
    D->io = (double*)io;
    D->x[0] = x0; D->x[1] = x1; D->F[0] = F0; D->F[1] = F1;
    D->b = b; D->d = d;
    D->x32[0] = (float*)x320; D->x32[1] = (float*)x321; D->b32 = (float*)b32; D->F32 = (float*)F32;
    D->rhs = rhs; D->w = w; D->V = V; D->part = (double*)part;
    D->P.eps64 = (const double*)e64; D->P.src64 = (const double*)s64;
    D->P.eps32 = (const float*)e32; D->P.src32 = (const float*)s32;
  }
  return off;
}

long long class_key(int pde, int pc, long long ncell) {
  int lg = 0;
  while ((1LL << lg) < ncell) ++lg;
  return ((long long)pde * 4 + pc) * 64 + lg;
}

}  // namespace

#define BK(call, what)                                                      \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      if (why) *why = std::string(what) + ": " + cudaGetErrorString(e_);    \
      return JFNK_E_CUDA;                                                   \
    }                                                                       \
  } while (0)

bool BatchEngine::supports(const jfnk_problem* pr, const jfnk_opts* o, std::string* why) {
  ProbDev P;
  if (!pr || !o) { if (why) *why = "null argument"; return false; }
  if (!make_probdev(pr, &P, why)) return false;
  int ts, tj;
  if (pair_of(o->prec, &ts, &tj) < 0) { if (why) *why = "batched solves run FP64, FP32 or mixed FP32"; return false; }
  if (o->krylov != JFNK_GMRES) { if (why) *why = "batched solves use GMRES"; return false; }
  if (o->lin != JFNK_AD && o->lin != JFNK_FD) { if (why) *why = "bad linearisation"; return false; }
  if (o->restart < 1 || o->restart > kMaxM) { if (why) *why = "restart out of range"; return false; }
  if (o->max_newton < 0 || o->max_krylov < 1) { if (why) *why = "bad iteration limits"; return false; }
  if (!(o->tol_newton >= 0) || !(o->tol_krylov >= 0)) { if (why) *why = "bad tolerances"; return false; }
  if (!(o->ls_min_alpha > 0.0 && o->ls_min_alpha <= 1.0)) { if (why) *why = "bad ls_min_alpha"; return false; }
  if (o->fd_rule != JFNK_EPS_SCALED && o->fd_rule != JFNK_EPS_PAPER) { if (why) *why = "bad fd_rule"; return false; }
  if (o->ortho != JFNK_CGS2 && o->ortho != JFNK_DCGS2) {
    if (why) *why = "batched solves use CGS2 or delayed CGS2 Arnoldi";
    return false;
  }
  if (pr->pde == JFNK_MAXWELL_VEC2D || o->precond != JFNK_PRECOND_NONE) {
    if (why) *why = "the vector Maxwell problem and its preconditioner run through jfnk_solve";
    return false;
  }
  return true;
}

size_t BatchEngine::workspace_bytes(const jfnk_problem* pr, const jfnk_opts* o) {
  std::string why;
  if (!supports(pr, o, &why)) return 0;
  return carve(pr, o, nullptr, nullptr);
}

BatchEngine::BatchEngine(int device) : device_(device) {
  cudaSetDevice(device);
  cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking);
  cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, device);
  if (nsm_ < 1) nsm_ = 1;
  for (int g = 0; g < kGroups; ++g) {
    cudaStreamCreateWithFlags(&side_[g], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&join_[g], cudaEventDisableTiming);
  }
  cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming);
  cudaMalloc((void**)&d_cnt_, kGroups * 2 * sizeof(unsigned int));
  cudaMemset(d_cnt_, 0, kGroups * 2 * sizeof(unsigned int));
}

BatchEngine::~BatchEngine() {
  cudaSetDevice(device_);
  cudaStreamSynchronize(stream_);
  for (Slot& s : slots_)
    if (s.ws) cudaFree(s.ws);
  if (exec_) cudaGraphExecDestroy(exec_);
  for (int g = 0; g < kGroups; ++g) {
    if (side_[g]) cudaStreamDestroy(side_[g]);
    if (join_[g]) cudaEventDestroy(join_[g]);
  }
  if (fork_) cudaEventDestroy(fork_);
  if (stream_) cudaStreamDestroy(stream_);
  cudaFree(d_desc_); cudaFree(d_flags_); cudaFree(d_items_); cudaFree(d_cnt_);
  if (h_flags_) cudaFreeHost(h_flags_);
  cudaGetLastError();
}

jfnk_status BatchEngine::grow(int cap, std::string* why) {
  if (cap <= cap_) return JFNK_OK;
  BK(cudaStreamSynchronize(stream_), "synchronize");
  BatDesc* nd = nullptr;
  int* nf = nullptr;
  int* nh = nullptr;
  BK(cudaMalloc((void**)&nd, (size_t)cap * sizeof(BatDesc)), "cudaMalloc");
  BK(cudaMalloc((void**)&nf, (size_t)cap * sizeof(int)), "cudaMalloc");
  BK(cudaHostAlloc((void**)&nh, (size_t)cap * sizeof(int), cudaHostAllocDefault), "cudaHostAlloc");
  BK(cudaMemset(nf, 0, (size_t)cap * sizeof(int)), "memset");
  std::memset(nh, 0, (size_t)cap * sizeof(int));
  if (cap_ > 0) {
    BK(cudaMemcpy(nd, d_desc_, (size_t)cap_ * sizeof(BatDesc), cudaMemcpyDeviceToDevice), "copy");
    BK(cudaMemcpy(nf, d_flags_, (size_t)cap_ * sizeof(int), cudaMemcpyDeviceToDevice), "copy");
  }
  cudaFree(d_desc_); cudaFree(d_flags_);
  if (h_flags_) cudaFreeHost(h_flags_);
  d_desc_ = nd; d_flags_ = nf; h_flags_ = nh;
  // descriptors hold a pointer to their done flag: repoint them
  for (int i = 0; i < cap_; ++i)
    if (slots_[i].used) {
      slots_[i].desc.done_flag = d_flags_ + i;
      BK(cudaMemcpy(d_desc_ + i, &slots_[i].desc, sizeof(BatDesc), cudaMemcpyHostToDevice), "copy");
    }
  slots_.resize(cap);
  cap_ = cap;
  dirty_ = true;
  return JFNK_OK;
}

jfnk_status BatchEngine::admit(const BatRequest& r, std::string* why) {
  if (!supports(&r.prob, &r.opts, why)) return JFNK_E_INVALID;
  ProbDev P;
  make_probdev(&r.prob, &P, why);
  if (!P.bvp && r.steps < 1) { if (why) *why = "steps must be >= 1"; return JFNK_E_INVALID; }
  if (!r.x0 || !r.x_out) { if (why) *why = "null state"; return JFNK_E_INVALID; }
  BK(cudaSetDevice(device_), "cudaSetDevice");
  int ts = 0, tj = 0;
  const int pc = pair_of(r.opts.prec, &ts, &tj);
  const int tc = tile_for(r.prob.pde, ts, tj, &r.prob, why);
  if (tc <= 0) return JFNK_E_CUDA;
  int slot = -1;
  for (int i = 0; i < cap_; ++i)
    if (!slots_[i].used) { slot = i; break; }
  if (slot < 0) {
    slot = cap_;
    jfnk_status s = grow(std::max(16, 2 * cap_), why);
    if (s) return s;
  }
  if (r.prob.pde * 3 + pc >= kGroups) { if (why) *why = "no batch group for this PDE"; return JFNK_E_INVALID; }
  Slot& S = slots_[slot];
  const size_t bytes = carve(&r.prob, &r.opts, nullptr, nullptr);
  void* ws = nullptr;
  BK(cudaMalloc(&ws, bytes), "cudaMalloc slot");
  BatDesc D;
  std::memset(&D, 0, sizeof(D));
  carve(&r.prob, &r.opts, (unsigned char*)ws, &D);
  const double* e64 = D.P.eps64; const double* s64 = D.P.src64;
  const float* e32 = D.P.eps32; const float* s32 = D.P.src32;
  D.P = P;
  D.P.eps64 = e64; D.P.src64 = s64; D.P.eps32 = e32; D.P.src32 = s32;
  D.N = P.ncell * P.nf;
  D.tc = tc;
  D.ntile = (int)((P.ncell + tc - 1) / tc);
  D.nunit = (int)((P.ncell + kBatUnit - 1) / kBatUnit);
  D.ts = ts; D.tj = tj;
  D.lin = r.opts.lin; D.fd_rule = r.opts.fd_rule; D.m = r.opts.restart;
  D.max_newton = r.opts.max_newton; D.max_krylov = r.opts.max_krylov;
  D.steps = P.bvp ? 1 : r.steps;
  D.born = (P.bvp && r.opts.born_start) ? 1 : 0;
  D.ortho = r.opts.ortho;
  D.tol_newton = r.opts.tol_newton; D.tol_krylov = r.opts.tol_krylov;
  D.fd_eps = r.opts.fd_eps; D.ls_c1 = r.opts.ls_c1; D.ls_min_alpha = r.opts.ls_min_alpha;
  D.done_flag = d_flags_ + slot;
  auto fail_free = [&](const char* what, cudaError_t e) {
    cudaFree(ws);
    if (why) *why = std::string(what) + ": " + cudaGetErrorString(e);
    return JFNK_E_CUDA;
  };
  cudaError_t e;
  // problem arrays (Maxwell), initial state, control state
  const long long nc = P.ncell;
  if (D.P.eps64) {
    if ((e = cudaMemcpyAsync((void*)D.P.eps64, r.prob.aux[0], nc * 8, cudaMemcpyDefault, stream_)) ||
        (e = launch_cast(VT_F64, VT_F32, nc, D.P.eps64, (void*)D.P.eps32, 1.0, stream_)))
      return fail_free("problem arrays", e);
  }
  if (D.P.src64) {
    if ((e = cudaMemcpyAsync((void*)D.P.src64, r.prob.aux[1], 2 * nc * 8, cudaMemcpyDefault, stream_)) ||
        (e = launch_cast(VT_F64, VT_F32, 2 * nc, D.P.src64, (void*)D.P.src32, 1.0, stream_)))
      return fail_free("problem arrays", e);
  }
  if ((e = cudaMemcpyAsync(D.io, r.x0, (size_t)D.N * 8, cudaMemcpyDefault, stream_))) return fail_free("copy in", e);
  BatState st;
  std::memset(&st, 0, sizeof(st));
  st.phase = PH_IN;
  st.stage = D.born ? 0 : 1;
  st.g.m = D.m;
  if ((e = cudaMemcpyAsync(D.st, &st, sizeof(st), cudaMemcpyHostToDevice, stream_)) ||
      (e = cudaMemsetAsync(d_flags_ + slot, 0, sizeof(int), stream_)) ||
      (e = cudaMemcpyAsync(d_desc_ + slot, &D, sizeof(D), cudaMemcpyHostToDevice, stream_)))
    return fail_free("admit", e);
  if ((e = cudaStreamSynchronize(stream_))) return fail_free("admit", e);   // host copies above are on the stack
  S.used = true;
  S.req = r;
  S.desc = D;
  S.ws = ws;
  S.bytes = bytes;
  S.group = r.prob.pde * 3 + pc;
  S.t0 = std::chrono::steady_clock::now();
  h_flags_[slot] = 0;
  bytes_ += bytes;
  n_active_ += 1;
  dirty_ = true;
  return JFNK_OK;
}

// Work lists of all groups and the graph: per group a chain of `launches_`
// batch-kernel launches; the groups' chains run as parallel branches.
jfnk_status BatchEngine::rebuild(std::string* why) {
  BK(cudaStreamSynchronize(stream_), "synchronize");
  std::vector<int2> items;
  int off[kGroups + 1];
  for (int g = 0; g < kGroups; ++g) {
    off[g] = (int)items.size();
    for (int i = 0; i < cap_; ++i) {
      const Slot& s = slots_[i];
      if (!s.used || s.group != g || h_flags_[i]) continue;
      for (int t = 0; t < s.desc.ntile; ++t) items.push_back(make_int2(i, t));
    }
  }
  off[kGroups] = (int)items.size();
  if ((int)items.size() > items_cap_) {
    cudaFree(d_items_);
    d_items_ = nullptr;
    items_cap_ = std::max<int>((int)items.size(), 2 * items_cap_);
    BK(cudaMalloc((void**)&d_items_, (size_t)items_cap_ * sizeof(int2)), "cudaMalloc items");
  }
  if (!items.empty())
    BK(cudaMemcpy(d_items_, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice), "copy items");
  if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; }
  graph_launches_ = 0;
  std::vector<int> groups;
  for (int g = 0; g < kGroups; ++g)
    if (off[g + 1] > off[g]) groups.push_back(g);
  if (groups.empty()) { dirty_ = false; return JFNK_OK; }
  cudaGraph_t graph = nullptr;
  BK(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t ce = cudaEventRecord(fork_, stream_);
  for (size_t q = 0; q < groups.size() && ce == cudaSuccess; ++q) {
    const int g = groups[q];
    cudaStream_t sg = (q == 0) ? stream_ : side_[g];
    if (q > 0) ce = cudaStreamWaitEvent(sg, fork_, 0);
    BatLaunch L;
    L.desc = d_desc_;
    L.items = d_items_ + off[g];
    L.nitems = off[g + 1] - off[g];
    L.next = d_cnt_ + 2 * g;
    L.ndone = d_cnt_ + 2 * g + 1;
    const int pde = g / 3, pc = g % 3;
    const int ts = pc == 1 ? VT_F32 : VT_F64, tj = pc == 0 ? VT_F64 : VT_F32;
    const int grid = std::min(L.nitems, batch_grid_cap(pde, ts, tj, nsm_));
    for (int l = 0; l < launches_ && ce == cudaSuccess; ++l) {
      ce = batch_launch(pde, ts, tj, L, grid, sg);
      graph_launches_ += 1;
    }
    if (q > 0 && ce == cudaSuccess) {
      ce = cudaEventRecord(join_[g], sg);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(stream_, join_[g], 0);
    }
  }
  cudaError_t ee = cudaStreamEndCapture(stream_, &graph);
  if (ce != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (why) *why = std::string("graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee);
    return JFNK_E_CUDA;
  }
  cudaError_t ie = cudaGraphInstantiate(&exec_, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    exec_ = nullptr;
    if (why) *why = std::string("graph instantiate: ") + cudaGetErrorString(ie);
    return JFNK_E_CUDA;
  }
  dirty_ = false;
  return JFNK_OK;
}

jfnk_status BatchEngine::finish(int i, BatResult* out, std::string* why) {
  Slot& s = slots_[i];
  BatState st;
  BK(cudaMemcpyAsync(&st, s.desc.st, sizeof(BatState), cudaMemcpyDeviceToHost, stream_), "copy out");
  BK(cudaMemcpyAsync(s.req.x_out, s.desc.io, (size_t)s.desc.N * 8, cudaMemcpyDefault, stream_), "copy out");
  BK(cudaStreamSynchronize(stream_), "synchronize");
  jfnk_report& rep = out->rep;
  std::memset(&rep, 0, sizeof(rep));
  rep.status = st.status;
  rep.steps_done = st.steps_done;
  rep.steps_failed = st.steps_failed;
  rep.newton_its = st.newton_its;
  rep.krylov_its = st.krylov_its;
  rep.jvp_calls = st.jvp_calls;
  rep.ls_backtracks = st.ls_backtracks;
  rep.ls_failures = st.ls_failures;
  rep.krylov_failures = st.krylov_failures;
  rep.res0 = st.res0;
  rep.res_final = st.res_final;
  rep.dt_last = st.dt;
  rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s.t0).count();
  out->tag = s.req.tag;
  out->status = (jfnk_status)st.first_bad;
  BK(cudaFree(s.ws), "cudaFree slot");
  bytes_ -= s.bytes;
  n_active_ -= 1;
  s.used = false;
  s.ws = nullptr;
  h_flags_[i] = 0;
  dirty_ = true;
  return JFNK_OK;
}

jfnk_status BatchEngine::advance(std::vector<BatResult>* finished, std::string* why) {
  BK(cudaSetDevice(device_), "cudaSetDevice");
  if (n_active_ == 0) return JFNK_OK;
  if (dirty_) {
    jfnk_status s = rebuild(why);
    if (s) return s;
  }
  if (exec_) {
    BK(cudaGraphLaunch(exec_, stream_), "graph launch");
    kernel_launches_ += graph_launches_;
  }
  BK(cudaMemcpyAsync(h_flags_, d_flags_, (size_t)cap_ * sizeof(int), cudaMemcpyDeviceToHost, stream_), "flags");
  BK(cudaStreamSynchronize(stream_), "synchronize");
  for (int i = 0; i < cap_; ++i) {
    if (!slots_[i].used || !h_flags_[i]) continue;
    BatResult r;
    jfnk_status s = finish(i, &r, why);
    if (s) return s;
    if (finished) finished->push_back(r);
  }
  return JFNK_OK;
}

int BatchEngine::tuned_tile(int pde, int prec, long long ncell) const {
  int ts, tj;
  const int pc = pair_of(prec, &ts, &tj);
  if (pc < 0) return 0;
  auto it = tiles_.find(class_key(pde, pc, ncell));
  return it == tiles_.end() ? 0 : it->second;
}

void BatchEngine::drop_all() {
  cudaSetDevice(device_);
  cudaStreamSynchronize(stream_);
  for (int i = 0; i < cap_; ++i) {
    Slot& s = slots_[i];
    if (!s.used) continue;
    cudaFree(s.ws);
    s.ws = nullptr;
    s.used = false;
    h_flags_[i] = 0;
  }
  n_active_ = 0;
  bytes_ = 0;
  dirty_ = true;
  cudaGetLastError();
}

// Cells per tile for a problem class, by measurement: a probe batch of
// solves of this size (about a million cells in all) runs the four phases of
// an Arnoldi step at j = 8 with each candidate tile size; the fastest is kept
// for the class (PDE, precision pair, size rounded up to a power of two).
// Results do not depend on the choice (reductions are per 256-cell unit).
int BatchEngine::tile_for(int pde, int ts, int tj, const jfnk_problem* prob, std::string* why) {
  const long long ncell = (long long)prob->nx * prob->ny;
  const int pc = ts == VT_F32 ? 1 : (tj == VT_F32 ? 2 : 0);
  const long long key = class_key(pde, pc, ncell);
  auto it = tiles_.find(key);
  if (it != tiles_.end()) return it->second;
  if (tile_override_ > 0) {
    tiles_[key] = tile_override_;
    return tile_override_;
  }
  std::vector<int> cands;
  for (int c : kTileCands)
    if (c == kBatUnit || (long long)c / 2 < ncell) cands.push_back(c);
  if (cands.size() == 1) { tiles_[key] = cands[0]; return cands[0]; }
  // probe solves: same problem shape, state 0.5, basis 0.01 (finite values; numbers are not used)
  jfnk_problem pr = *prob;
  pr.aux[0] = nullptr; pr.aux[1] = nullptr;
  jfnk_opts o;
  jfnk_default_opts(&o, pc == 0 ? JFNK_FP64 : (pc == 1 ? JFNK_FP32 : JFNK_MIXED_FP32));
  o.restart = 16;
  ProbDev P;
  if (!make_probdev(&pr, &P, why)) return -1;
  const int R = (int)std::max<long long>(1, std::min<long long>(64, (1LL << 20) / ncell));
  const size_t bytes = carve(&pr, &o, nullptr, nullptr);
  std::vector<void*> ws(R, nullptr);
  BatDesc* dd = nullptr;
  int* dflag = nullptr;
  int2* ditems = nullptr;
  unsigned int* dcnt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = cands[0];
  auto cleanup = [&]() {
    cudaStreamSynchronize(stream_);
    for (void* p : ws) cudaFree(p);
    cudaFree(dd); cudaFree(dflag); cudaFree(ditems); cudaFree(dcnt);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
  };
  auto err = [&](const char* what, cudaError_t e) {
    if (why) *why = std::string("tile tuning: ") + what + ": " + cudaGetErrorString(e);
    cleanup();
    return -1;
  };
  cudaError_t e;
  if ((e = cudaMalloc((void**)&dd, R * sizeof(BatDesc))) || (e = cudaMalloc((void**)&dflag, R * sizeof(int))) ||
      (e = cudaMalloc((void**)&dcnt, 2 * sizeof(unsigned int))) || (e = cudaMemset(dcnt, 0, 2 * sizeof(unsigned int))) ||
      (e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1)))
    return err("setup", e);
  std::vector<BatDesc> hd(R);
  const long long N = P.ncell * P.nf;
  const std::vector<double> half((size_t)N, 0.5);
  for (int r = 0; r < R; ++r) {
    if ((e = cudaMalloc(&ws[r], bytes))) return err("cudaMalloc", e);
    BatDesc& D = hd[r];
    std::memset(&D, 0, sizeof(D));
    carve(&pr, &o, (unsigned char*)ws[r], &D);
    D.P = P;
    D.N = N;
    D.nunit = (int)((P.ncell + kBatUnit - 1) / kBatUnit);
    D.ts = ts; D.tj = tj; D.lin = JFNK_AD; D.m = o.restart;
    D.max_newton = 1; D.max_krylov = 1; D.steps = 1;
    D.done_flag = dflag + r;
    // state 0.5 and basis 0.01 through the cast kernel from a constant FP64 buffer
    if ((e = cudaMemcpy(D.io, half.data(), (size_t)N * 8, cudaMemcpyHostToDevice)) ||
        (e = launch_cast(VT_F64, ts, N, D.io, D.x[0], 1.0, stream_)) ||
        (e = launch_cast(VT_F64, tj, N, D.io, D.w, 1.0, stream_)))
      return err("probe init", e);
    if (ts != tj && (e = launch_cast(VT_F64, VT_F32, N, D.io, D.x32[0], 1.0, stream_))) return err("probe init", e);
    for (int t = 0; t < 9; ++t)
      if ((e = launch_cast(VT_F64, tj, N, D.io, (char*)D.V + (size_t)t * N * vt_size(tj), 0.02, stream_)))
        return err("probe init", e);
    BatState st;
    std::memset(&st, 0, sizeof(st));
    st.phase = PH_JVP;
    st.stage = 2;
    st.j = 8;
    st.g.m = o.restart;
    for (int t = 0; t <= kMaxM; ++t) st.g.scale[t] = 1.0;
    for (int t = 0; t <= 8; ++t) { st.g.h1[t] = 1e-3; st.g.h2[t] = 1e-3; }
    if ((e = cudaMemcpy(D.st, &st, sizeof(st), cudaMemcpyHostToDevice))) return err("probe state", e);
  }
  float best_ms = 1e30f;
  for (int c : cands) {
    std::vector<int2> items;
    for (int r = 0; r < R; ++r) {
      hd[r].tc = c;
      hd[r].ntile = (int)((P.ncell + c - 1) / c);
      for (int t = 0; t < hd[r].ntile; ++t) items.push_back(make_int2(r, t));
    }
    cudaFree(ditems);
    ditems = nullptr;
    if ((e = cudaMalloc((void**)&ditems, items.size() * sizeof(int2))) ||
        (e = cudaMemcpy(ditems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(dd, hd.data(), R * sizeof(BatDesc), cudaMemcpyHostToDevice)))
      return err("probe items", e);
    BatLaunch L;
    L.desc = dd; L.items = ditems; L.nitems = (int)items.size(); L.next = dcnt; L.ndone = dcnt + 1;
    const int grid = std::min(L.nitems, batch_grid_cap(pde, ts, tj, nsm_));
    for (int l = 0; l < 4; ++l)
      if ((e = batch_launch(pde, ts, tj, L, grid, stream_))) return err("probe launch", e);
    if ((e = cudaEventRecord(e0, stream_))) return err("event", e);
    for (int l = 0; l < 8; ++l)
      if ((e = batch_launch(pde, ts, tj, L, grid, stream_))) return err("probe launch", e);
    if ((e = cudaEventRecord(e1, stream_)) || (e = cudaEventSynchronize(e1))) return err("event", e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cleanup();
  tiles_[key] = best;
  return best;
}

}  // namespace jfnk
