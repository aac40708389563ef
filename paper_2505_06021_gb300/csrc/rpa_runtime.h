// Host runtime state of an rpa_ctx: executors (stream + workspace + pinned
// staging), the batched-launch cache and the serving scheduler.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rpa.h"
#include "rpa_internal.h"

namespace rpa {

// Growable pinned host buffer.
struct HostStage {
  void* ptr = nullptr;
  size_t bytes = 0;
  bool reserve(size_t n) {
    if (n <= bytes) return true;
    release();
    size_t want = n < 4096 ? 4096 : n;
    if (cudaHostAlloc(&ptr, want, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return false;
    }
    bytes = want;
    return true;
  }
  void release() {
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
  }
};

// One independent execution lane: its own streams, events, device workspace
// and pinned host buffers.  A synchronous entry point uses the context's
// default lane; the serving scheduler runs each admitted job on a lane of its
// own so that jobs overlap on the device.
struct Exec {
  cudaStream_t s = nullptr;   // compute
  cudaStream_t cs = nullptr;  // host -> device staging copies
  cudaEvent_t ready[2] = {nullptr, nullptr};
  cudaEvent_t freed[2] = {nullptr, nullptr};
  cudaEvent_t done = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // per-kernel timing: (class, start, end) recorded on the launching stream
  struct Mark {
    int cls, n;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t take_event();
  HostStage hstage;  // uploads (tables)
  HostStage hbin;    // uploads (tables of the frequency-batched chi0)
  HostStage hres;    // downloads: [int status | pad | Ec | eps[nqw] | parts[2 nqw]]
  bool init();
  void destroy();
  bool ensure_ws(size_t bytes);
  int& status_word() { return *reinterpret_cast<int*>(hres.ptr); }
  double* results() { return reinterpret_cast<double*>(reinterpret_cast<char*>(hres.ptr) + 64); }
};

// The frequency-batched chi0 of one job: the plan and every q's tables
// (their images in the lane's pinned buffer hbin).
struct BinJob {
  bool on = false;
  FreqPlan plan;
  std::vector<BinQHost> qh;  // per q
  int Kt_max = 0, np_max = 0;
  size_t meta_bytes = 0;  // the pinned image block (doubles, then every q's ints)
};

struct ServeState;  // serving.cu
struct BatchCache;  // batch.cu

}  // namespace rpa

struct rpa_ctx {
  int device = 0;
  int n_slices = 4;
  size_t cap = 0;
  double timeout_s = 60.0;
  int max_inflight = 64;
  int chi0_freq = 0;  // rpa_config.chi0_freq
  rpa::Exec ex;  // default lane for the synchronous entry points
  std::atomic<uint64_t> launches{0};
  std::mutex mu;  // serialises the synchronous entry points on this context
  std::mutex err_mu;
  std::string last_error;
  rpa::ServeState* serve = nullptr;
  rpa::BatchCache* batch = nullptr;
  bool prof = false;
  double prof_ms[RPA_K_COUNT] = {0};
  uint64_t prof_n[RPA_K_COUNT] = {0};
  uint64_t flops0 = 0;                 // process-wide tensor flops at rpa_profile(ctx, 1)
  std::atomic<uint64_t> h2d_bytes{0};  // host -> device staging bytes since then
};

namespace rpa {

// Workspace of one lane for a job processed in q-batches of qb q-points.
struct Layout {
  size_t meta, dtab, chi, T, L, Vc, stageC, stageV, eps, mixed, ao, binmeta, total;
  size_t slice_cap;  // mixed path: bytes for the weighted operand's digit planes
  int qb;            // q per staging batch (d table, host staging, AO coefficients)
  int qt;            // q per tail batch (chi, L, Vc, T: V factor and log-det)
};

// Device pointers into a lane's workspace.
struct Bufs {
  const void** Cptrs;  // [n_q*n_k]
  int* kidx;           // [n_q*n_k]
  int* kqidx;          // [n_q*n_k]
  double* omega;       // [n_w]
  double* zeta_w;      // [n_w]
  double* w_q;         // [n_q]
  double* Ec;          // [1]
  double* eps;         // [n_q*n_w]
  double* parts;       // [n_q*n_w*2]
  double* ldV;         // [n_q] ln det V(q) (inverse-form tail)
  int* status;
  double* dtab;
  double* chi;
  double* T;
  double* L;
  double* Vc;  // copy of V(q) for Tr(chi V) (inverse-form tail), else null
  char* stageC[2];
  char* stageV[2];
  double* eps_occ;
  double* eps_virt;
  void* mixed;
  size_t mixed_bytes;
  size_t slice_cap;
  char* ao;       // AO-form jobs: fit table, half-transforms, one q's C (ao_internal.h)
  char* binmeta;  // frequency-batched chi0: the job's bin tables, or null
};

void ctx_set_error(rpa_ctx* ctx, const char* fmt, ...);
rpa_status validate_job(const rpa_job* j, char* msg, size_t len);
size_t job_footprint(const rpa_job* j, int n_slices, size_t ws_cap);
// Device workspace a lane needs for the job (part of job_footprint).
size_t job_workspace(const rpa_job* j, int n_slices, size_t ws_cap);
// Enqueues the whole hot path of `job` on lane `ex` (no host wait) and records
// ex.done after the results were copied into ex.hres.
// allow_bin: use the frequency-batched chi0 when the context's setting and
// the job's plan allow it (the synchronous entry point; serving lanes do not).
rpa_status energy_enqueue(rpa_ctx* ctx, Exec& ex, const rpa_job* job, size_t ws_cap, bool allow_bin = false);
// After ex.done has completed: decodes the device status and copies results.
rpa_status energy_finish(rpa_ctx* ctx, Exec& ex, const rpa_job* job, double* Ec, double* eps_qw, double* parts);
// Bounded wait for an event (RPA_E_TIMEOUT after timeout_s).
rpa_status wait_event(rpa_ctx* ctx, cudaEvent_t ev, double timeout_s);
// Timing marks around kernel launches (no-ops when profiling is off or ex is
// null); prof_collect adds the elapsed times of completed marks to the
// context's totals and recycles the events.
void prof_begin(rpa_ctx* ctx, Exec* ex, cudaStream_t s);
void prof_end(rpa_ctx* ctx, Exec* ex, cudaStream_t s, int cls, int n_kernels);
void prof_collect(rpa_ctx* ctx, Exec* ex);
// mixed_ws: include the split-precision chi0 workspace (a batch supplies its own).
// qt: q per tail batch (0: qt = qb).  bj: the job's frequency-batched chi0, if any.
Layout plan_layout(const rpa_job* j, int qb, int n_slices, size_t ws_cap, bool mixed_ws, int qt = 0,
                   const BinJob* bj = nullptr);
int choose_qb(const rpa_job* j, int n_slices, size_t cap, const BinJob* bj = nullptr);
int choose_qt(const rpa_job* j, int qb, int n_slices, size_t cap, const BinJob* bj = nullptr);
// Builds the frequency-batched plan of a split-precision job (band energies
// read back from the device when they live there) and its per-q tables in
// ex.hbin; bj.on stays false when the context turns it off or it saves nothing.
rpa_status bin_job_build(rpa_ctx* ctx, Exec& ex, const rpa_job* j, BinJob& bj);
Bufs carve(void* ws, const rpa_job* j, const Layout& L);
size_t sync_ws_cap(rpa_ctx* ctx);
size_t tables_bytes(const rpa_job* j);
void fill_tables_host(const rpa_job* j, const void* const* Cdev, char* h);
rpa_status enqueue_table_copies(rpa_ctx* ctx, const rpa_job* j, const Bufs& b, const char* h, cudaStream_t s);
rpa_status stage_dtab(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                      const double* eps_occ, const double* eps_virt, cudaStream_t s);
// V-side work of the tail: V copies, V = LL^H (and, for the inverse form,
// ln det V and -V^-1).
rpa_status stage_vside(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                       const void* const* Vdev, cudaStream_t s);
rpa_status stage_tail(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                      const void* const* Vdev, cudaStream_t s);
rpa_status decode_status(rpa_ctx* ctx, int st, int n_w);
void serving_shutdown(rpa_ctx* ctx);
void batch_release(rpa_ctx* ctx);
}  // namespace rpa
