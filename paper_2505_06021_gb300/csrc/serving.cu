// Serving runtime: continuous batching of RPA energy jobs on one GB300.
//
// rpa_submit() deep-copies a job's host descriptors into a pending queue.  A
// scheduler thread admits pending jobs in arrival order while the device
// memory they account for stays under the context's HBM cap: the inputs of the
// running jobs plus every lane's workspace (lanes keep their workspace between
// jobs; idle lanes give theirs back when a new job would not fit otherwise),
// and while fewer than max_inflight jobs run.  An
// admitted job gets an execution lane of its own (stream, workspace, pinned
// buffers) and its whole hot path is enqueued there at once, so the kernels of
// all running jobs share the device; the scheduler polls the lanes' completion
// events, publishes results and admits the next jobs as soon as memory frees
// up.  The paper's analogue is the (q, omega) group decomposition of Sec. 2.6
// (independent work units, one gather of the results); here the independent
// units are whole jobs and the gather is the per-ticket result table.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "rpa_runtime.h"

namespace rpa {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeJob {
  uint64_t ticket = 0;
  rpa_job job{};
  std::vector<int> pair_k, pair_kq;
  std::vector<double> w_q, omega, zeta_w;
  std::vector<const void*> C, V;
  size_t footprint = 0;  // inputs + workspace
  size_t ws_need = 0;    // workspace part
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = 0;  // 0 pending, 1 running, 2 done
  rpa_status status = RPA_OK;
  double Ec = 0;
  std::vector<double> eps;
  Exec* lane = nullptr;
  std::string error;
};

struct ServeState {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<ServeJob>> pending;
  std::vector<std::shared_ptr<ServeJob>> running;
  std::map<uint64_t, std::shared_ptr<ServeJob>> tickets;
  std::vector<std::unique_ptr<Exec>> lanes;
  std::vector<Exec*> free_lanes;
  size_t inputs_used = 0;  // device inputs of the running jobs
  size_t ws_total = 0;     // workspace held by all lanes
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  std::vector<double> lat, wait;
  uint64_t done = 0;
  size_t max_pending = 4096;
  int peak_running = 0;     // most jobs on the device at once
  size_t peak_used = 0;     // largest inputs_used + ws_total
};

static size_t ws_alloc_size(size_t need) { return std::max(need, (size_t)64 << 20); }

// A free lane for a job that needs `need` bytes of workspace: the smallest
// free lane that already holds enough, else the free lane holding the most
// (its workspace will be reallocated), else a new lane (nullptr if none could
// be made).  *extra: growth of the lanes' total workspace if this lane runs
// the job.
static Exec* pick_lane(ServeState* S, size_t need, size_t* extra) {
  int best = -1;
  for (int i = 0; i < (int)S->free_lanes.size(); ++i) {
    const size_t b = S->free_lanes[i]->ws_bytes;
    if (b >= need && (best < 0 || b < S->free_lanes[best]->ws_bytes)) best = i;
  }
  if (best < 0)
    for (int i = 0; i < (int)S->free_lanes.size(); ++i)
      if (best < 0 || S->free_lanes[i]->ws_bytes > S->free_lanes[best]->ws_bytes) best = i;
  Exec* e = nullptr;
  if (best >= 0) {
    e = S->free_lanes[best];
  } else {
    std::unique_ptr<Exec> n(new Exec());
    if (!n->init()) {
      n->destroy();
      return nullptr;
    }
    S->lanes.push_back(std::move(n));
    e = S->lanes.back().get();
    S->free_lanes.push_back(e);
  }
  *extra = e->ws_bytes >= need ? 0 : ws_alloc_size(need) - e->ws_bytes;
  return e;
}

// Gives back the workspace of idle lanes other than `keep` until `want` bytes
// were released or none is left; returns the bytes released.
static size_t release_idle(ServeState* S, Exec* keep, size_t want) {
  size_t freed = 0;
  for (Exec* e : S->free_lanes) {
    if (freed >= want) break;
    if (e == keep || !e->ws) continue;
    cudaStreamSynchronize(e->s);
    cudaFree(e->ws);
    freed += e->ws_bytes;
    S->ws_total -= e->ws_bytes;
    e->ws = nullptr;
    e->ws_bytes = 0;
  }
  return freed;
}

static size_t lane_ws_cap(rpa_ctx* ctx) { return std::min<size_t>(ctx->cap / 4, (size_t)24 << 30); }

static void scheduler(rpa_ctx* ctx) {
  ServeState* S = ctx->serve;
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progress = false;
    // 1. admit in arrival order while memory and slots allow
    while (!S->pending.empty() && (int)S->running.size() < ctx->max_inflight) {
      std::shared_ptr<ServeJob> j = S->pending.front();
      size_t extra = 0;
      Exec* lane = pick_lane(S, j->ws_need, &extra);
      const size_t inputs = j->footprint - j->ws_need;
      if (lane) {
        size_t total = S->inputs_used + inputs + S->ws_total + extra;
        if (total > ctx->cap) total -= release_idle(S, lane, total - ctx->cap);
        // the first job always runs (its footprint alone is below the cap)
        if (total > ctx->cap && !S->running.empty()) break;
      }
      S->pending.pop_front();
      j->t_admit = now_s();
      if (!lane) {
        j->status = RPA_E_CUDA;
        j->error = "cannot create an execution lane";
        j->state = 2;
        j->t_done = now_s();
        progress = true;
        continue;
      }
      // memory the caller holds outside the cap (its own tensors) can leave
      // the device short: give back idle workspace before this lane grows
      if (extra > 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b < extra + ((size_t)1 << 30))
          release_idle(S, lane, extra + ((size_t)1 << 30) - free_b);
      }
      S->free_lanes.erase(std::find(S->free_lanes.begin(), S->free_lanes.end(), lane));
      j->lane = lane;
      j->state = 1;
      S->inputs_used += inputs;
      S->ws_total += extra;
      S->running.push_back(j);
      S->peak_running = std::max(S->peak_running, (int)S->running.size());
      S->peak_used = std::max(S->peak_used, S->inputs_used + S->ws_total);
      lk.unlock();
      rpa_status st = energy_enqueue(ctx, *lane, &j->job, lane_ws_cap(ctx));
      lk.lock();
      if (st != RPA_OK) {
        j->status = st;
        j->error = ctx->last_error;
        // let the lane drain whatever was enqueued before the failure
        cudaEventRecord(lane->done, lane->s);
        j->Ec = 0;
      }
      progress = true;
    }
    // 2. collect finished jobs
    for (size_t i = 0; i < S->running.size();) {
      std::shared_ptr<ServeJob> j = S->running[i];
      cudaError_t e = cudaEventQuery(j->lane->done);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (j->status == RPA_OK) {
        if (e != cudaSuccess) {
          j->status = RPA_E_CUDA;
          j->error = cudaGetErrorString(e);
        } else {
          j->eps.resize((size_t)j->job.n_q * j->job.n_w);
          j->status = energy_finish(ctx, *j->lane, &j->job, &j->Ec, j->eps.data(), nullptr);
          if (j->status) j->error = ctx->last_error;
        }
      }
      j->t_done = now_s();
      j->state = 2;
      S->inputs_used -= j->footprint - j->ws_need;
      S->free_lanes.push_back(j->lane);
      j->lane = nullptr;
      S->lat.push_back(j->t_done - j->t_submit);
      S->wait.push_back(j->t_admit - j->t_submit);
      S->done++;
      S->running.erase(S->running.begin() + i);
      progress = true;
    }
    if (progress) S->cv.notify_all();
    if (S->stop && S->pending.empty() && S->running.empty()) break;
    if (!progress) {
      if (S->running.empty() && S->pending.empty())
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
      else
        S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

static ServeState* ensure_serving(rpa_ctx* ctx) {
  if (!ctx->serve) {
    ctx->serve = new ServeState();
    ctx->serve->th = std::thread(scheduler, ctx);
  }
  return ctx->serve;
}

void serving_shutdown(rpa_ctx* ctx) {
  ServeState* S = ctx->serve;
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  for (auto& l : S->lanes) l->destroy();
  delete S;
  ctx->serve = nullptr;
}

static double pct(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double r = p * (v.size() - 1);
  const size_t lo = (size_t)r, hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (r - lo) * (v[hi] - v[lo]);
}

}  // namespace rpa

using namespace rpa;

extern "C" {

rpa_status rpa_submit(rpa_ctx* ctx, const rpa_job* job, uint64_t* ticket) {
  if (!ctx || !ticket) return RPA_E_INVAL;
  char msg[512];
  if (validate_job(job, msg, sizeof msg)) {
    ctx_set_error(ctx, "%s", msg);
    return RPA_E_INVAL;
  }
  std::shared_ptr<ServeJob> j(new ServeJob());
  const size_t npk = (size_t)job->n_q * job->n_k;
  j->pair_k.assign(job->pair_k, job->pair_k + npk);
  j->pair_kq.assign(job->pair_kq, job->pair_kq + npk);
  j->w_q.assign(job->w_q, job->w_q + job->n_q);
  j->omega.assign(job->omega, job->omega + job->n_w);
  j->zeta_w.assign(job->zeta_w, job->zeta_w + job->n_w);
  j->C.assign(job->C, job->C + npk);
  j->V.assign(job->V, job->V + job->n_q);
  j->job = *job;
  j->job.pair_k = j->pair_k.data();
  j->job.pair_kq = j->pair_kq.data();
  j->job.w_q = j->w_q.data();
  j->job.omega = j->omega.data();
  j->job.zeta_w = j->zeta_w.data();
  j->job.C = j->C.data();
  j->job.V = j->V.data();
  j->footprint = job_footprint(job, ctx->n_slices, lane_ws_cap(ctx));
  j->ws_need = job_workspace(job, ctx->n_slices, lane_ws_cap(ctx));
  if (j->footprint > ctx->cap) {
    ctx_set_error(ctx, "job footprint %zu bytes exceeds the HBM cap %zu", j->footprint, ctx->cap);
    return RPA_E_NOMEM;
  }
  ServeState* S = ensure_serving(ctx);
  std::lock_guard<std::mutex> g(S->mu);
  if (S->pending.size() >= S->max_pending) {
    ctx_set_error(ctx, "request queue full (%zu pending)", S->pending.size());
    return RPA_E_BUSY;
  }
  j->ticket = S->next_ticket++;
  j->t_submit = now_s();
  S->pending.push_back(j);
  S->tickets[j->ticket] = j;
  *ticket = j->ticket;
  S->cv.notify_all();
  return RPA_OK;
}

rpa_status rpa_poll(rpa_ctx* ctx, uint64_t ticket, double* Ec, double* eps_qw) {
  if (!ctx || !ctx->serve) return RPA_E_INVAL;
  ServeState* S = ctx->serve;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) {
    ctx_set_error(ctx, "unknown ticket %llu", (unsigned long long)ticket);
    return RPA_E_INVAL;
  }
  std::shared_ptr<ServeJob> j = it->second;
  if (j->state != 2) return RPA_E_NOTREADY;
  S->tickets.erase(it);
  if (j->status != RPA_OK) {
    ctx_set_error(ctx, "job %llu: %s", (unsigned long long)ticket, j->error.c_str());
    return j->status;
  }
  if (Ec) *Ec = j->Ec;
  if (eps_qw) std::copy(j->eps.begin(), j->eps.end(), eps_qw);
  return RPA_OK;
}

rpa_status rpa_wait(rpa_ctx* ctx, uint64_t ticket, double timeout_s, double* Ec, double* eps_qw) {
  if (!ctx || !ctx->serve) return RPA_E_INVAL;
  ServeState* S = ctx->serve;
  const double t0 = now_s();
  {
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
      auto it = S->tickets.find(ticket);
      if (it == S->tickets.end()) break;
      if (it->second->state == 2) break;
      const double left = timeout_s - (now_s() - t0);
      if (left <= 0) {
        ctx_set_error(ctx, "rpa_wait: ticket %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
        return RPA_E_TIMEOUT;
      }
      S->cv.wait_for(lk, std::chrono::microseconds((long)std::min(left * 1e6, 2000.0)));
    }
  }
  return rpa_poll(ctx, ticket, Ec, eps_qw);
}

rpa_status rpa_serving_stats(rpa_ctx* ctx, uint64_t* jobs_done, double* lat_mean, double* lat_p50, double* lat_p99,
                             double* wait_p50, double* wait_p99) {
  if (!ctx) return RPA_E_INVAL;
  if (!ctx->serve) {
    if (jobs_done) *jobs_done = 0;
    if (lat_mean) *lat_mean = 0;
    if (lat_p50) *lat_p50 = 0;
    if (lat_p99) *lat_p99 = 0;
    if (wait_p50) *wait_p50 = 0;
    if (wait_p99) *wait_p99 = 0;
    return RPA_OK;
  }
  ServeState* S = ctx->serve;
  std::lock_guard<std::mutex> g(S->mu);
  double m = 0;
  for (double v : S->lat) m += v;
  if (jobs_done) *jobs_done = S->done;
  if (lat_mean) *lat_mean = S->lat.empty() ? 0.0 : m / S->lat.size();
  if (lat_p50) *lat_p50 = pct(S->lat, 0.50);
  if (lat_p99) *lat_p99 = pct(S->lat, 0.99);
  if (wait_p50) *wait_p50 = pct(S->wait, 0.50);
  if (wait_p99) *wait_p99 = pct(S->wait, 0.99);
  return RPA_OK;
}

rpa_status rpa_serving_peak(rpa_ctx* ctx, int* max_running, size_t* max_bytes) {
  if (!ctx) return RPA_E_INVAL;
  int r = 0;
  size_t b = 0;
  if (ctx->serve) {
    std::lock_guard<std::mutex> g(ctx->serve->mu);
    r = ctx->serve->peak_running;
    b = ctx->serve->peak_used;
  }
  if (max_running) *max_running = r;
  if (max_bytes) *max_bytes = b;
  return RPA_OK;
}

}  // extern "C"
