// serve.cu -- the request server of jfnk_submit / jfnk_poll (see serve.h).
#include "serve.h"

#include <chrono>
#include <cstring>

namespace jfnk {

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Server::Server(int device, size_t budget, int slots) : device_(device), budget_(budget) {
  if (slots < 1) slots = 1;
  for (int s = 0; s < slots; ++s) threads_.emplace_back(&Server::worker, this, s);
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
  const size_t need = workspace_estimate(prob, opts);
  if (need == 0) return JFNK_E_INVALID;
  if (budget_ && need > budget_) return JFNK_E_OOM;
  Req* r = new Req();
  r->prob = *prob;
  r->opts = *opts;
  r->x0 = x0;
  r->x_out = x_out;
  r->steps = steps;
  r->need = need;
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

void Server::worker(int slot) {
  (void)slot;
  jfnk_ctx* ctx = nullptr;
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] {
        if (stop_) return true;
        if (queue_.empty()) return false;
        return budget_ == 0 || reserved_ + queue_.front()->need <= budget_;
      });
      if (stop_) break;
      r = queue_.front();
      queue_.pop_front();
      reserved_ += r->need;
      r->state = 1;
    }
    jfnk_status s = JFNK_OK;
    if (!ctx) s = jfnk_create(&ctx, device_, 0, nullptr);
    jfnk_report rep;
    std::memset(&rep, 0, sizeof(rep));
    if (s == JFNK_OK) s = jfnk_set_problem(ctx, &r->prob);
    if (s == JFNK_OK) s = jfnk_solve(ctx, &r->opts, r->x0, r->x_out, r->steps, &rep);
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
  if (ctx) jfnk_destroy(ctx);
}

}  // namespace jfnk
