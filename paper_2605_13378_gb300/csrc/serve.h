// serve.h -- continuous-batching request server behind jfnk_submit / jfnk_poll.
//
// Requests enter a FIFO queue and are admitted when their workspace fits in
// the HBM budget left by the requests already running. Two executors take
// them:
// * the batch engine (one thread): requests it supports (GMRES; FP64, FP32
//   or mixed FP32) up to a size limit join the running batch between two
//   replays of its launch graph, so a request that arrives while others run
//   starts within one replay and shares every kernel launch with them;
// * slot workers (one context and stream each) run the other requests (and
//   larger ones, for which the single-solve kernels stream the basis at HBM
//   speed) through jfnk_solve, concurrently with the batch.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "jfnk.h"

namespace jfnk {

// Device bytes jfnk_solve allocates for this problem and these options.
size_t workspace_estimate(const jfnk_problem* prob, const jfnk_opts* opts);

class Server {
 public:
  Server(int device, size_t budget, int slots);
  ~Server();
  jfnk_status submit(const jfnk_problem* prob, const jfnk_opts* opts, const double* x0, double* x_out, int steps,
                     unsigned long long* ticket);
  jfnk_status poll(unsigned long long ticket, jfnk_report* rep);

 private:
  struct Req {
    unsigned long long id;
    jfnk_problem prob;
    jfnk_opts opts;
    const double* x0;
    double* x_out;
    int steps;
    size_t need;
    bool batched;          // runs in the batch engine
    int state;             // 0 queued, 1 running, 2 done
    jfnk_status status;
    jfnk_report rep;
    double t_submit;
  };
  void worker(int slot);
  void batch_worker();
  void complete(Req* r, jfnk_status s, const jfnk_report& rep);
  int device_;
  size_t budget_, reserved_ = 0;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Req*> queue_;
  std::map<unsigned long long, Req*> reqs_;
  unsigned long long next_id_ = 1;
  bool stop_ = false;
  std::vector<std::thread> threads_;
  long long batch_max_cells_ = 0;   // largest problem (cells x fields) routed to the batch engine
};

}  // namespace jfnk
