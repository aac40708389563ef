// Serving runtime: continuous batching of RPA energy jobs on one GB300.
//
// rpa_submit() deep-copies a job's host descriptors into a pending queue.  A
// scheduler thread admits pending jobs in arrival order while the device
// memory it accounts for stays under the context's HBM cap: the inputs of the
// running jobs plus every lane's workspace (lanes keep their workspace between
// jobs; idle lanes give theirs back when a new batch would not fit otherwise),
// and while fewer than max_inflight jobs run.  The device-resident jobs that
// are waiting when a lane frees up are admitted together as one micro-batch:
// their (q, omega) work runs through the batch engine (shared persistent
// tensor-core launches over all their (job, q) segments, per-job tail work on
// side streams, one ragged log-det launch), so small jobs fill the GPU
// together; micro-batches on different lanes overlap on the device.  Jobs
// with inputs in host memory (staged copies) and jobs too large to hold every
// q's workspace at once run alone on a lane, q-batch by q-batch.  The
// scheduler polls the lanes' completion events, publishes results and admits
// the next jobs as soon as memory frees up.  The paper's analogue is the
// (q, omega) group decomposition of Sec. 2.6 (independent work units, one
// gather of the results).
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch_internal.h"
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
  bool batchable = false;  // device-resident and small enough to share a micro-batch
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = 0;  // 0 pending, 1 running, 2 done
  rpa_status status = RPA_OK;
  double Ec = 0;
  std::vector<double> eps;
  std::string error;
};

// An execution lane: stream, workspace and pinned buffers (Exec) plus side
// streams for the batch engine's tail work.
struct ServeLane {
  Exec ex;
  SideStreams side;
};

// Jobs admitted together and running on one lane.
struct ServeBatch {
  std::vector<std::shared_ptr<ServeJob>> jobs;
  std::vector<rpa_job> desc;    // their descriptors, in batch order
  std::unique_ptr<Plan> plan;   // null: a single host-memory job (energy_enqueue)
  ServeLane* lane = nullptr;
  size_t inputs = 0;
  bool failed = false;          // enqueue failed: every job reports `error`
  rpa_status status = RPA_OK;
  std::string error;
};

struct ServeState {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<ServeJob>> pending;
  std::vector<std::unique_ptr<ServeBatch>> running;
  int running_jobs = 0;
  std::map<uint64_t, std::shared_ptr<ServeJob>> tickets;
  std::vector<std::unique_ptr<ServeLane>> lanes;
  std::vector<ServeLane*> free_lanes;
  size_t inputs_used = 0;  // device inputs of the running jobs
  size_t ws_total = 0;     // workspace held by all lanes
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  std::vector<double> lat, wait;
  uint64_t done = 0;
  size_t max_pending = 4096;
  int peak_running = 0;     // most jobs on the device at once
  int peak_batch = 0;       // most jobs admitted as one micro-batch
  size_t peak_used = 0;     // largest inputs_used + ws_total
};

static size_t ws_alloc_size(size_t need) { return std::max(need, (size_t)64 << 20); }

static size_t lanes_ws(ServeState* S) {
  size_t t = 0;
  for (const auto& l : S->lanes) t += l->ex.ws_bytes;
  return t;
}

// Jobs per micro-batch (each (job, q) is a segment of the shared launches).
constexpr int kMaxBatch = 32;
// Micro-batches in flight at once: arrivals while all lanes are busy wait and
// are admitted together when one frees up.
constexpr int kMaxLanes = 4;

// A free lane for `need` bytes of workspace: the smallest free lane that
// already holds enough, else the free lane holding the most (its workspace
// will be reallocated), else a new lane (nullptr if none could be made).
// *extra: growth of the lanes' total workspace if this lane is used.
static ServeLane* pick_lane(ServeState* S, size_t need, size_t* extra) {
  int best = -1;
  for (int i = 0; i < (int)S->free_lanes.size(); ++i) {
    const size_t b = S->free_lanes[i]->ex.ws_bytes;
    if (b >= need && (best < 0 || b < S->free_lanes[best]->ex.ws_bytes)) best = i;
  }
  if (best < 0)
    for (int i = 0; i < (int)S->free_lanes.size(); ++i)
      if (best < 0 || S->free_lanes[i]->ex.ws_bytes > S->free_lanes[best]->ex.ws_bytes) best = i;
  ServeLane* l = nullptr;
  if (best >= 0) {
    l = S->free_lanes[best];
  } else if ((int)S->lanes.size() >= kMaxLanes) {
    return nullptr;  // all lanes busy
  } else {
    std::unique_ptr<ServeLane> n(new ServeLane());
    if (!n->ex.init() || !n->side.init()) {
      n->side.release();
      n->ex.destroy();
      return nullptr;
    }
    S->lanes.push_back(std::move(n));
    l = S->lanes.back().get();
    S->free_lanes.push_back(l);
  }
  *extra = l->ex.ws_bytes >= need ? 0 : ws_alloc_size(need) - l->ex.ws_bytes;
  return l;
}

// Gives back the workspace of idle lanes other than `keep` until `want` bytes
// were released or none is left; returns the bytes released.
static size_t release_idle(ServeState* S, ServeLane* keep, size_t want) {
  size_t freed = 0;
  for (ServeLane* l : S->free_lanes) {
    if (freed >= want) break;
    Exec* e = &l->ex;
    if (l == keep || !e->ws) continue;
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
    // 1. admit in arrival order while memory and slots allow: the waiting
    //    device-resident jobs as one micro-batch per free lane
    while (!S->pending.empty() && S->running_jobs < ctx->max_inflight) {
      std::unique_ptr<ServeBatch> B(new ServeBatch());
      const bool alone = !S->pending.front()->batchable;
      size_t ws_need = 0;
      if (alone) {
        B->jobs.push_back(S->pending.front());
        ws_need = B->jobs[0]->ws_need;
        B->inputs = B->jobs[0]->footprint - B->jobs[0]->ws_need;
        B->desc.push_back(B->jobs[0]->job);
      } else {
        // greedy prefix of the queue: device jobs whose inputs and workspace
        // fit next to what runs; the plan then gives the batch's workspace
        size_t est = 0;
        for (const std::shared_ptr<ServeJob>& j : S->pending) {
          if (!j->batchable || (int)B->jobs.size() >= kMaxBatch ||
              S->running_jobs + (int)B->jobs.size() >= ctx->max_inflight)
            break;
          const size_t add = j->footprint;
          if (!B->jobs.empty() && S->inputs_used + S->ws_total + est + add > ctx->cap) break;
          B->jobs.push_back(j);
          est += add;
          B->inputs += j->footprint - j->ws_need;
        }
        for (const auto& j : B->jobs) B->desc.push_back(j->job);
        B->plan = batch_plan(B->desc.data(), (int)B->desc.size(), ctx->n_slices, lane_ws_cap(ctx));
        ws_need = B->plan->ws_bytes;
      }
      size_t extra = 0;
      ServeLane* lane = pick_lane(S, ws_need, &extra);
      if (!lane && (int)S->lanes.size() >= kMaxLanes) break;  // wait for a lane
      if (lane) {
        size_t total = S->inputs_used + B->inputs + S->ws_total + extra;
        if (total > ctx->cap) total -= release_idle(S, lane, total - ctx->cap);
        // the estimate admitted too much: shrink the batch from its end
        while (total > ctx->cap && B->jobs.size() > 1) {
          B->inputs -= B->jobs.back()->footprint - B->jobs.back()->ws_need;
          B->jobs.pop_back();
          B->desc.pop_back();
          B->plan = batch_plan(B->desc.data(), (int)B->desc.size(), ctx->n_slices, lane_ws_cap(ctx));
          ws_need = B->plan->ws_bytes;
          lane = pick_lane(S, ws_need, &extra);
          if (!lane) break;  // the lane was free a moment ago: cannot happen, but stay safe
          total = S->inputs_used + B->inputs + S->ws_total + extra;
        }
        // a single job always runs when nothing else does (its footprint is below the cap)
        if (lane && total > ctx->cap && !S->running.empty()) break;
      }
      const double t_admit = now_s();
      for (size_t k = 0; k < B->jobs.size(); ++k) S->pending.pop_front();
      if (!lane) {
        for (auto& j : B->jobs) {
          j->t_admit = t_admit;
          j->status = RPA_E_CUDA;
          j->error = "cannot create an execution lane";
          j->state = 2;
          j->t_done = now_s();
        }
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
      for (auto& j : B->jobs) {
        j->t_admit = t_admit;
        j->state = 1;
      }
      B->lane = lane;
      S->inputs_used += B->inputs;
      S->ws_total += extra;
      S->running_jobs += (int)B->jobs.size();
      S->peak_running = std::max(S->peak_running, S->running_jobs);
      S->peak_batch = std::max(S->peak_batch, (int)B->jobs.size());
      S->peak_used = std::max(S->peak_used, S->inputs_used + S->ws_total);
      ServeBatch* Bp = B.get();
      S->running.push_back(std::move(B));
      lk.unlock();
      rpa_status st = RPA_OK;
      bool no_memory = false;
      if (!Bp->plan) {
        st = energy_enqueue(ctx, lane->ex, &Bp->jobs[0]->job, lane_ws_cap(ctx));
      } else if (!lane->ex.ensure_ws(Bp->plan->ws_bytes) || !lane->ex.hstage.reserve(Bp->plan->pin_bytes + 64)) {
        ctx_set_error(ctx, "cannot allocate the serving batch's workspace");
        st = RPA_E_NOMEM;
        no_memory = true;
      } else {
        char* pin = (char*)lane->ex.hstage.ptr;
        batch_fill_tables(*Bp->plan, Bp->desc.data(), (int)Bp->desc.size(), pin);
        uint64_t nk = 0;
        st = batch_enqueue(ctx, lane->side, *Bp->plan, Bp->desc.data(), (char*)lane->ex.ws, pin, lane->ex.s, false,
                           &nk, nullptr);
        if (st == RPA_OK && cudaEventRecord(lane->ex.done, lane->ex.s) != cudaSuccess) st = RPA_E_CUDA;
      }
      lk.lock();
      if (no_memory) S->ws_total = lanes_ws(S);  // the lane may have given up its old workspace
      if (no_memory && S->running.size() > 1) {
        // the device is short (memory held outside the cap): put the jobs back
        // at the head of the queue and admit again when a running batch ends
        for (size_t k = Bp->jobs.size(); k-- > 0;) {
          Bp->jobs[k]->state = 0;
          S->pending.push_front(Bp->jobs[k]);
        }
        S->inputs_used -= Bp->inputs;
        S->running_jobs -= (int)Bp->jobs.size();
        S->free_lanes.push_back(lane);
        S->running.pop_back();
        break;
      }
      if (st != RPA_OK) {
        Bp->failed = true;
        Bp->status = st;
        Bp->error = ctx->last_error;
        // let the lane drain whatever was enqueued before the failure
        cudaEventRecord(lane->ex.done, lane->ex.s);
      }
      progress = true;
    }
    // 2. collect finished batches
    for (size_t i = 0; i < S->running.size();) {
      ServeBatch* B = S->running[i].get();
      cudaError_t e = cudaEventQuery(B->lane->ex.done);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const double t_done = now_s();
      for (size_t k = 0; k < B->jobs.size(); ++k) {
        ServeJob* j = B->jobs[k].get();
        if (B->failed) {
          j->status = B->status;
          j->error = B->error;
        } else if (e != cudaSuccess) {
          j->status = RPA_E_CUDA;
          j->error = cudaGetErrorString(e);
        } else if (!B->plan) {
          j->eps.resize((size_t)j->job.n_q * j->job.n_w);
          j->status = energy_finish(ctx, B->lane->ex, &j->job, &j->Ec, j->eps.data(), nullptr);
          if (j->status) j->error = ctx->last_error;
        } else {
          const char* r = (const char*)B->lane->ex.hstage.ptr + B->plan->jobs[k].res_off;
          int sw;
          memcpy(&sw, r, sizeof sw);
          j->status = decode_status(ctx, sw, j->job.n_w);
          if (j->status) {
            j->error = ctx->last_error;
          } else {
            const size_t nqw = (size_t)j->job.n_q * j->job.n_w;
            memcpy(&j->Ec, r + 64, sizeof(double));
            j->eps.resize(nqw);
            memcpy(j->eps.data(), r + 64 + sizeof(double), sizeof(double) * nqw);
          }
        }
        j->t_done = t_done;
        j->state = 2;
        S->lat.push_back(j->t_done - j->t_submit);
        S->wait.push_back(j->t_admit - j->t_submit);
        S->done++;
      }
      S->inputs_used -= B->inputs;
      S->running_jobs -= (int)B->jobs.size();
      S->free_lanes.push_back(B->lane);
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
  for (auto& l : S->lanes) {
    l->side.release();
    l->ex.destroy();
  }
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
  if (job->ao) {
    ctx_set_error(ctx, "rpa_submit: AO-form jobs are run with rpa_energy");
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
  if (job->mem == RPA_MEM_DEVICE) {
    // the batch engine holds every q's split-precision workspace at once:
    // jobs whose batch workspace stays within a lane's cap share micro-batches,
    // larger ones run alone q-batch by q-batch
    const size_t inputs = j->footprint - j->ws_need;
    const size_t ws_b = batch_plan(&j->job, 1, ctx->n_slices, lane_ws_cap(ctx))->ws_bytes;
    if (ws_b <= lane_ws_cap(ctx)) {
      j->batchable = true;
      j->ws_need = ws_b;
      j->footprint = inputs + ws_b;
    }
  }
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

rpa_status rpa_serving_peak(rpa_ctx* ctx, int* max_running, size_t* max_bytes, int* max_batch) {
  if (!ctx) return RPA_E_INVAL;
  int r = 0, mb = 0;
  size_t b = 0;
  if (ctx->serve) {
    std::lock_guard<std::mutex> g(ctx->serve->mu);
    r = ctx->serve->peak_running;
    b = ctx->serve->peak_used;
    mb = ctx->serve->peak_batch;
  }
  if (max_running) *max_running = r;
  if (max_bytes) *max_bytes = b;
  if (max_batch) *max_batch = mb;
  return RPA_OK;
}

}  // extern "C"
