// batch_engine.h -- host side of the batched solver: admits solves into
// device slots, keeps the (solve, tile) work lists and a captured CUDA graph
// of batch-kernel launches, replays it, and hands back finished solves.
// Used by jfnk_solve_batch and by the request server. Internal.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <map>
#include <string>
#include <vector>

#include "batch.h"
#include "jfnk.h"

namespace jfnk {

struct BatRequest {
  jfnk_problem prob;
  jfnk_opts opts;
  const double* x0;      // FP64 initial state (host or device), N entries
  double* x_out;         // FP64 result (host or device), N entries
  int steps;
  unsigned long long tag;
};

struct BatResult {
  unsigned long long tag;
  jfnk_status status;    // first non-OK status of the solve's Newton solves, else OK
  jfnk_report rep;
};

class BatchEngine {
 public:
  // The engine works on a CUDA stream of its own.
  explicit BatchEngine(int device);
  ~BatchEngine();
  BatchEngine(const BatchEngine&) = delete;
  BatchEngine& operator=(const BatchEngine&) = delete;

  // Whether the engine runs this problem with these options (GMRES, FP64 /
  // FP32 / mixed FP32, restart 1..64); why says what is not supported.
  static bool supports(const jfnk_problem* prob, const jfnk_opts* opts, std::string* why);
  // Device bytes a slot of this request holds while it runs.
  static size_t workspace_bytes(const jfnk_problem* prob, const jfnk_opts* opts);

  // Allocate the slot, copy the initial state in and queue the solve; it
  // starts with the next advance().
  jfnk_status admit(const BatRequest& r, std::string* why);
  // Replay the launch graph once (`launches` phases of every unfinished
  // solve), then collect the solves that finished: their results are copied
  // to x_out and their slots freed.
  jfnk_status advance(std::vector<BatResult>* finished, std::string* why);
  // Free every slot without finishing its solve (after an error).
  void drop_all();
  int active() const { return n_active_; }
  size_t bytes_in_use() const { return bytes_; }
  // Tile size the autotuner chose for a problem class (cells per tile).
  int tile_for(int pde, int ts, int tj, const jfnk_problem* prob, std::string* why);
  // The tile size chosen for a class so far (0: not tuned yet).
  int tuned_tile(int pde, int prec, long long ncell) const;
  // Cells per tile for classes not tuned yet (0: measure per class).
  void set_tile_override(int cells) { tile_override_ = cells; }
  void set_launches_per_replay(int l) { launches_ = l < 1 ? 1 : l; dirty_ = true; }
  int launches_per_replay() const { return launches_; }
  long long kernel_launches() const { return kernel_launches_; }

 private:
  struct Slot {
    bool used = false;
    BatRequest req;
    BatDesc desc;
    void* ws = nullptr;
    size_t bytes = 0;
    int group = 0;
    std::chrono::steady_clock::time_point t0;
  };
  static constexpr int kGroups = 15;    // 5 PDEs (jfnk_pde) x 3 precision pairs
  jfnk_status rebuild(std::string* why);
  jfnk_status grow(int cap, std::string* why);
  jfnk_status finish(int slot, BatResult* out, std::string* why);

  int device_;
  cudaStream_t stream_ = nullptr;
  cudaStream_t side_[kGroups] = {};
  cudaEvent_t fork_ = nullptr, join_[kGroups] = {};
  int nsm_ = 0;
  int launches_ = 48;
  std::vector<Slot> slots_;
  int cap_ = 0;
  BatDesc* d_desc_ = nullptr;
  int* d_flags_ = nullptr;              // per slot: 1 once the solve is done
  int* h_flags_ = nullptr;              // pinned copy
  int2* d_items_ = nullptr;
  int items_cap_ = 0;
  unsigned int* d_cnt_ = nullptr;       // per group: work counter, CTAs done
  int n_active_ = 0;
  size_t bytes_ = 0;
  bool dirty_ = true;
  cudaGraphExec_t exec_ = nullptr;
  long long kernel_launches_ = 0;
  int graph_launches_ = 0;              // kernel launches in one replay
  std::map<long long, int> tiles_;      // autotuned cells per tile, by problem class
  int tile_override_ = 0;               // fixed cells per tile for untuned classes (0: none)
};

}  // namespace jfnk
