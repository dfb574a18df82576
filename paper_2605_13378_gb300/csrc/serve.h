// serve.h -- continuous-batching request server behind jfnk_submit / jfnk_poll.
//
// Requests enter a FIFO queue. A request is admitted when one of the
// server's slots is free and its workspace estimate fits in the HBM budget
// left by the requests already running; each slot owns a context and a CUDA
// stream, so admitted solves run concurrently on the device and a request
// that arrives while others run starts as soon as a slot and memory free up.
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
    int state;             // 0 queued, 1 running, 2 done
    jfnk_status status;
    jfnk_report rep;
    double t_submit;
  };
  void worker(int slot);
  int device_;
  size_t budget_, reserved_ = 0;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Req*> queue_;
  std::map<unsigned long long, Req*> reqs_;
  unsigned long long next_id_ = 1;
  bool stop_ = false;
  std::vector<std::thread> threads_;
};

}  // namespace jfnk
