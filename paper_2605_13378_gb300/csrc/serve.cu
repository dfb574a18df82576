// serve.cu -- the request server of jfnk_submit / jfnk_poll (see serve.h).
#include "serve.h"

#include <chrono>
#include <cstdlib>
#include <cstring>
#include <string>

#include "batch_engine.h"

namespace jfnk {

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Server::Server(int device, size_t budget, int slots) : device_(device), budget_(budget) {
  if (slots < 1) slots = 1;
  batch_max_cells_ = 1LL << 20;   // unknowns (cells x fields) of the largest batched request
  for (int s = 0; s < slots; ++s) threads_.emplace_back(&Server::worker, this, s);
  threads_.emplace_back(&Server::batch_worker, this);
}

Server::~Server() {
  {
    std::lock_guard<std::mutex> lk(mu_);
    stop_ = true;
  }
  cv_.notify_all();
  for (auto& t : threads_) t.join();
  for (auto& kv : reqs_) delete kv.second;
  for (Req* r : queue_) (void)r;   // queued requests are owned by reqs_
}

jfnk_status Server::submit(const jfnk_problem* prob, const jfnk_opts* opts, const double* x0, double* x_out,
                           int steps, unsigned long long* ticket) {
  const long long cells = (long long)prob->nx * prob->ny *
                          pde_nfields(prob->pde);
  const bool batched = cells <= batch_max_cells_ && BatchEngine::supports(prob, opts, nullptr) &&
                       (prob->pde == JFNK_MAXWELL_TE2D || prob->pde == JFNK_MAXWELL_VEC2D || steps >= 1);
  const size_t need = batched ? BatchEngine::workspace_bytes(prob, opts) : workspace_estimate(prob, opts);
  if (need == 0) return JFNK_E_INVALID;
  if (budget_ && need > budget_) return JFNK_E_OOM;
  Req* r = new Req();
  r->prob = *prob;
  r->opts = *opts;
  r->x0 = x0;
  r->x_out = x_out;
  r->steps = steps;
  r->need = need;
  r->batched = batched;
  r->state = 0;
  r->status = JFNK_E_BUSY;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(mu_);
    r->id = next_id_++;
    reqs_[r->id] = r;
    queue_.push_back(r);
    *ticket = r->id;
  }
  cv_.notify_all();
  return JFNK_OK;
}

jfnk_status Server::poll(unsigned long long ticket, jfnk_report* rep) {
  std::lock_guard<std::mutex> lk(mu_);
  auto it = reqs_.find(ticket);
  if (it == reqs_.end()) return JFNK_E_INVALID;
  Req* r = it->second;
  if (r->state != 2) return JFNK_E_BUSY;
  if (rep) *rep = r->rep;
  const jfnk_status s = r->status;
  reqs_.erase(it);
  delete r;
  return s;
}

void Server::complete(Req* r, jfnk_status s, const jfnk_report& rep0) {
  jfnk_report rep = rep0;
  rep.status = s;
  rep.ms = now_ms() - r->t_submit;   // latency: submit to completion
  {
    std::lock_guard<std::mutex> lk(mu_);
    r->rep = rep;
    r->status = s;
    r->state = 2;
    reserved_ -= r->need;
  }
  cv_.notify_all();
}

void Server::worker(int slot) {
  (void)slot;
  jfnk_ctx* ctx = nullptr;
  for (;;) {
    Req* r = nullptr;
    {
      // the oldest queued request for a slot worker, once its workspace fits the budget
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] {
        if (stop_) return true;
        for (Req* q : queue_)
          if (!q->batched) return budget_ == 0 || reserved_ + q->need <= budget_;
        return false;
      });
      if (stop_) break;
      for (auto it = queue_.begin(); it != queue_.end(); ++it)
        if (!(*it)->batched) { r = *it; queue_.erase(it); break; }
      reserved_ += r->need;
      r->state = 1;
    }
    jfnk_status s = JFNK_OK;
    if (!ctx) s = jfnk_create(&ctx, device_, 0, nullptr);
    jfnk_report rep;
    std::memset(&rep, 0, sizeof(rep));
    if (s == JFNK_OK) s = jfnk_set_problem(ctx, &r->prob);
    if (s == JFNK_OK) s = jfnk_solve(ctx, &r->opts, r->x0, r->x_out, r->steps, &rep);
    complete(r, s, rep);
  }
  if (ctx) jfnk_destroy(ctx);
}

// The batch engine's thread: admit every queued batched request whose
// workspace fits (oldest first), replay the launch graph once, hand back the
// solves that finished, repeat; sleep while there is nothing to run.
void Server::batch_worker() {
  BatchEngine* eng = nullptr;
  std::vector<Req*> adm;
  std::vector<BatResult> fin;
  std::string why;
  for (;;) {
    adm.clear();
    {
      std::unique_lock<std::mutex> lk(mu_);
      auto ready = [&] {
        for (Req* q : queue_)
          if (q->batched && (budget_ == 0 || reserved_ + q->need <= budget_)) return true;
        return false;
      };
      const bool busy = eng && eng->active() > 0;
      if (!busy) cv_.wait(lk, [&] { return stop_ || ready(); });
      if (stop_) break;
      for (auto it = queue_.begin(); it != queue_.end();) {
        Req* q = *it;
        if (q->batched && (budget_ == 0 || reserved_ + q->need <= budget_)) {
          reserved_ += q->need;
          q->state = 1;
          adm.push_back(q);
          it = queue_.erase(it);
        } else {
          ++it;
        }
      }
    }
    if (!eng) {
      cudaSetDevice(device_);
      eng = new BatchEngine(device_);
    }
    for (Req* q : adm) {
      BatRequest br;
      br.prob = q->prob;
      br.opts = q->opts;
      br.x0 = q->x0;
      br.x_out = q->x_out;
      br.steps = q->steps;
      br.tag = q->id;
      const jfnk_status s = eng->admit(br, &why);
      if (s != JFNK_OK) {
        jfnk_report rep;
        std::memset(&rep, 0, sizeof(rep));
        complete(q, s, rep);
      }
    }
    fin.clear();
    const jfnk_status s = eng->advance(&fin, &why);
    if (s != JFNK_OK) {
      // a device error: every request in the batch fails with it
      std::vector<Req*> lost;
      {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto& kv : reqs_)
          if (kv.second->batched && kv.second->state == 1) lost.push_back(kv.second);
      }
      eng->drop_all();
      jfnk_report rep;
      std::memset(&rep, 0, sizeof(rep));
      for (Req* q : lost) complete(q, s, rep);
      continue;
    }
    for (const BatResult& b : fin) {
      Req* q = nullptr;
      {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = reqs_.find(b.tag);
        if (it != reqs_.end()) q = it->second;
      }
      if (q) complete(q, b.status, b.rep);
    }
  }
  delete eng;
}

}  // namespace jfnk
