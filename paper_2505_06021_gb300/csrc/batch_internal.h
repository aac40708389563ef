// Batch engine shared by rpa_energy_batch and the serving scheduler: a plan
// lays out many jobs' workspace (in groups under a memory budget) and pinned
// staging; batch_enqueue issues the whole batch on a stream: tables and d
// tables, shared persistent tensor-core launches for the split-precision
// jobs, per-job tail work forked onto side streams, ragged log-det, the
// quadratures and the result copies into pinned memory.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "rpa_runtime.h"

namespace rpa {

struct JobPlan {
  Layout L;        // whole job in one q-batch, without the chi0 mixed region
  size_t ws_off;   // within the group's region
  size_t tab_off;  // pinned tables
  size_t res_off;  // pinned results: [status | pad to 64 | Ec | eps | parts]
  size_t mixed;    // mixed-path workspace of all its q
};

struct Group {
  int j0, j1;        // job range
  size_t mixed_off;  // shared mixed workspace of the group's q
  size_t mixed_bytes;
  size_t task_off;   // device ragged log-det task tables (complex, then real)
  size_t pin_task;   // their pinned staging
  int n_task_c, n_task_r;
  size_t bytes;
};

struct Plan {
  std::vector<uint64_t> sig;
  std::vector<JobPlan> jobs;
  std::vector<Group> groups;
  size_t ws_bytes = 0, pin_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernels per replay
  double work = 0.0;     // chi0 flops, for the wait limit
  ~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// Side streams for the per-job tail work, with fork/join events.
struct SideStreams {
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  bool ok = false;
  bool init();
  void release();
};

// Plan for n jobs; groups of jobs whose workspace fits `budget`.
std::unique_ptr<Plan> batch_plan(const rpa_job* jobs, int n, int n_slices, size_t budget);
// Writes every job's small tables into the pinned buffer (tables_bytes each).
void batch_fill_tables(const Plan& p, const rpa_job* jobs, int n, char* pin);
// Issues the batch on `s` (tables already filled); results land in `pin` at
// jobs[i].res_off: int status at +0, then (Ec, eps[n_q n_w], parts[2 n_q n_w])
// at +64.  tune: time split-K candidates (never under stream capture).
rpa_status batch_enqueue(rpa_ctx* ctx, SideStreams& side, const Plan& p, const rpa_job* jobs, char* ws, char* pin,
                         cudaStream_t s, bool tune, uint64_t* n_kernels, Exec* pex);

}  // namespace rpa
