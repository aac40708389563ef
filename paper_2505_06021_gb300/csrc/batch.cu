// Batched execution of many independent, uneven jobs in one call
// (rpa_energy_batch).
//
// The jobs are cut into groups whose workspace fits the context's HBM cap.  Per group, on
// the context's stream:
//   1. every job's small tables are copied in from pinned host memory and its
//      d_t(omega) table is built for all of its q;
//   2. chi0 of every (job, q) of the group's mixed-precision jobs runs in
//      shared persistent tensor-core launches (one per round of frequency
//      groups; each (job, q) is a segment of the launch), FP64 jobs run the
//      FP64 chi0 kernel;
//   3. every job runs its FP64 tail (V factor, sandwich, Cholesky log-det)
//      and the quadrature, and its results are copied to pinned host memory.
// The first call with a new batch signature (shapes, precisions, the device
// pointers that kernels take by value) runs eagerly, with the split-K
// autotuner timing its candidates, and then captures the same sequence into a
// CUDA graph; later calls with that signature refresh the pinned tables and
// replay the graph.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "batch_internal.h"
#include "rpa_internal.h"
#include "rpa_runtime.h"

namespace rpa {

#define CKB(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      ctx_set_error(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RPA_E_CUDA;                                                                              \
    }                                                                                                 \
  } while (0)

namespace {

constexpr size_t kBatchSliceCap = (size_t)4 << 30;  // digit planes of one q's weighted operand

BatchGeom geom_q(const rpa_job& j) {
  return BatchGeom{j.is_complex, j.n_aux, j.n_occ, j.n_virt, j.n_occ * j.n_virt, j.n_k, j.n_w, 1};
}

size_t a64(size_t x) { return (x + 63) & ~(size_t)63; }
size_t a1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

std::vector<uint64_t> signature(const rpa_job* jobs, int n, int n_slices) {
  std::vector<uint64_t> s;
  s.push_back((uint64_t)n);
  s.push_back((uint64_t)n_slices);
  for (int i = 0; i < n; ++i) {
    const rpa_job& j = jobs[i];
    s.push_back((uint64_t)j.is_complex | ((uint64_t)j.prec << 8) | ((uint64_t)j.mem << 16));
    s.push_back(((uint64_t)j.n_aux << 32) | (uint32_t)j.n_occ);
    s.push_back(((uint64_t)j.n_virt << 32) | (uint32_t)j.n_q);
    s.push_back(((uint64_t)j.n_k << 32) | (uint32_t)j.n_w);
    s.push_back((uint64_t)j.n_kpts);
    uint64_t z;
    memcpy(&z, &j.zeta_k, sizeof z);
    s.push_back(z);
    s.push_back((uint64_t)(uintptr_t)j.eps_occ);
    s.push_back((uint64_t)(uintptr_t)j.eps_virt);
    for (int q = 0; q < j.n_q; ++q) s.push_back((uint64_t)(uintptr_t)j.V[q]);
  }
  return s;
}

}  // namespace

std::unique_ptr<Plan> batch_plan(const rpa_job* jobs, int n, int n_slices, size_t budget) {
  std::unique_ptr<Plan> p(new Plan);
  p->jobs.resize(n);
  size_t pin = 0;
  for (int i = 0; i < n; ++i) {
    JobPlan& jp = p->jobs[i];
    jp.L = plan_layout(&jobs[i], jobs[i].n_q, n_slices, 0, false);
    jp.mixed = 0;
    if (jobs[i].prec == RPA_PREC_MIXED) {
      const size_t per_q = a1k(mixed_workspace_bytes(geom_q(jobs[i]), n_slices, kBatchSliceCap));
      jp.mixed = per_q * (size_t)jobs[i].n_q;
    }
    jp.tab_off = pin;
    pin += a64(tables_bytes(&jobs[i]));
    jp.res_off = pin;
    pin += 64 + a64(sizeof(double) * (1 + 3 * (size_t)jobs[i].n_q * jobs[i].n_w));
    const double nq = jobs[i].n_q, nk = jobs[i].n_k, nw = jobs[i].n_w;
    p->work += 8.0 * jobs[i].n_aux * (double)jobs[i].n_aux * jobs[i].n_occ * jobs[i].n_virt * nq * nk * nw;
  }
  // greedy groups in job order under the workspace budget
  int i = 0;
  while (i < n) {
    Group g{i, i, 0, 0, 0, 0, 0, 0, 0};
    size_t fp = 0, mx = 0;
    while (g.j1 < n) {
      const JobPlan& jp = p->jobs[g.j1];
      const size_t f2 = fp + a1k(jp.L.total), m2 = mx + jp.mixed;
      if (g.j1 > g.j0 && f2 + m2 + 1024 > budget) break;
      p->jobs[g.j1].ws_off = fp;
      fp = f2;
      mx = m2;
      ++g.j1;
    }
    for (int k = g.j0; k < g.j1; ++k)
      if (jobs[k].prec == RPA_PREC_MIXED) (jobs[k].is_complex ? g.n_task_c : g.n_task_r) += jobs[k].n_q * jobs[k].n_w;
    const size_t tbytes = a1k(sizeof(CholTask) * (size_t)(g.n_task_c + g.n_task_r));
    g.mixed_off = fp;
    g.mixed_bytes = mx ? mx + 1024 : 0;
    g.task_off = fp + g.mixed_bytes;
    g.pin_task = pin;
    pin += tbytes;
    g.bytes = g.task_off + tbytes;
    p->ws_bytes = std::max(p->ws_bytes, g.bytes);
    p->groups.push_back(g);
    i = g.j1;
  }
  p->pin_bytes = pin;
  return p;
}

bool SideStreams::init() {
  if (ok) return true;
  for (int k = 0; k < kSide; ++k) {
    if (cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming) != cudaSuccess) return false;
  }
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return false;
  ok = true;
  return true;
}

void SideStreams::release() {
  for (int k = 0; k < kSide; ++k) {
    if (side[k]) {
      cudaStreamSynchronize(side[k]);
      cudaStreamDestroy(side[k]);
    }
    if (join[k]) cudaEventDestroy(join[k]);
    side[k] = nullptr;
    join[k] = nullptr;
  }
  if (fork) cudaEventDestroy(fork);
  fork = nullptr;
  ok = false;
}

// The batch runs on the context's own stream (rpa_stream) with a workspace
// and pinned buffers of its own, kept between calls for graph replay.
struct BatchCache {
  Exec mem;  // workspace only (no streams)
  HostStage pin;
  std::unique_ptr<Plan> plan;
  SideStreams side;
};

void batch_release(rpa_ctx* ctx) {
  if (!ctx->batch) return;
  if (ctx->ex.s) cudaStreamSynchronize(ctx->ex.s);
  ctx->batch->side.release();
  ctx->batch->plan.reset();
  ctx->batch->pin.release();
  ctx->batch->mem.destroy();
  delete ctx->batch;
  ctx->batch = nullptr;
}

// Fills the pinned tables of every job (read by the upload copies when they
// execute).
void batch_fill_tables(const Plan& p, const rpa_job* jobs, int n, char* pin) {
  for (int i = 0; i < n; ++i) fill_tables_host(&jobs[i], jobs[i].C, pin + p.jobs[i].tab_off);
}

// Enqueues the whole batch on `s` (pinned tables already filled); *n_kernels
// gets the number of kernels enqueued.  pex (profiling lane, may be null)
// receives per-kernel-class timing marks; never set under stream capture.
rpa_status batch_enqueue(rpa_ctx* ctx, SideStreams& bc, const Plan& p, const rpa_job* jobs, char* ws, char* pin,
                         cudaStream_t s, bool tune, uint64_t* n_kernels, Exec* pex) {
  uint64_t nk = 0;
  struct HookCtx {
    rpa_ctx* ctx;
    Exec* ex;
  } hc{ctx, pex};
  const LaunchHook hook{&hc,
                        [](void* u, cudaStream_t st) {
                          HookCtx* h = (HookCtx*)u;
                          prof_begin(h->ctx, h->ex, st);
                        },
                        [](void* u, cudaStream_t st, int cls, int n) {
                          HookCtx* h = (HookCtx*)u;
                          prof_end(h->ctx, h->ex, st, cls, n);
                        }};
  const uint64_t l0 = ctx->launches.load();
  std::vector<Bufs> B(jobs ? p.jobs.size() : 0);
  for (const Group& g : p.groups) {
    for (int i = g.j0; i < g.j1; ++i) {
      B[i] = carve(ws + p.jobs[i].ws_off, &jobs[i], p.jobs[i].L);
      if (rpa_status st = enqueue_table_copies(ctx, &jobs[i], B[i], pin + p.jobs[i].tab_off, s)) return st;
      if (rpa_status st = stage_dtab(ctx, pex, &jobs[i], B[i], 0, jobs[i].n_q, jobs[i].eps_occ,
                                     jobs[i].eps_virt, s))
        return st;
    }
    std::vector<MixedQ> mq;
    int* mstatus = nullptr;
    for (int i = g.j0; i < g.j1; ++i) {
      const rpa_job& j = jobs[i];
      const size_t es = j.is_complex ? 16 : 8;
      const size_t NN = (size_t)j.n_aux * j.n_aux;
      const BatchGeom g1 = geom_q(j);
      if (j.prec == RPA_PREC_MIXED) {
        if (!mstatus) mstatus = B[i].status;
        for (int q = 0; q < j.n_q; ++q)
          mq.push_back(MixedQ{g1, (const double* const*)(B[i].Cptrs + (size_t)q * j.n_k),
                              B[i].dtab + (size_t)q * j.n_k * j.n_w * g1.n_ov,
                              B[i].chi + (size_t)q * j.n_w * NN * (es / 8), kBatchSliceCap});
      } else {
        BatchGeom ga = g1;
        ga.n_qb = j.n_q;
        prof_begin(ctx, pex, s);
        CKB(launch_chi0_fp64(ga, (const double* const*)B[i].Cptrs, B[i].dtab, B[i].chi, s));
        prof_end(ctx, pex, s, RPA_K_CHI0, 1);
        ctx->launches++;
      }
    }
    if (!mq.empty()) {
      uint64_t nl = 0;
      CKB(launch_chi0_mixed_multi(mq.data(), (int)mq.size(), ctx->n_slices, ws + g.mixed_off, g.mixed_bytes, mstatus,
                                  &nl, s, tune, pex ? &hook : nullptr));
      ctx->launches += nl;
    }
    // fork: per-job tail work on the side streams, largest jobs first.  FP64
    // jobs run their whole tail (sandwich form) there; mixed jobs only the
    // V-side work (V = LL^H, ln det V, -V^-1), their log-dets follow as one
    // ragged launch over all of the group's matrices.
    CKB(cudaEventRecord(bc.fork, s));
    const int nside = std::min(SideStreams::kSide, g.j1 - g.j0);
    for (int k = 0; k < nside; ++k) CKB(cudaStreamWaitEvent(bc.side[k], bc.fork, 0));
    std::vector<int> order;
    for (int i = g.j0; i < g.j1; ++i) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
      const double wa = (double)jobs[a].n_aux * jobs[a].n_aux * jobs[a].n_aux * jobs[a].n_q * jobs[a].n_w;
      const double wc = (double)jobs[c].n_aux * jobs[c].n_aux * jobs[c].n_aux * jobs[c].n_q * jobs[c].n_w;
      return wa > wc;
    });
    auto finish_job = [&](int i, cudaStream_t ss) -> rpa_status {
      const rpa_job& j = jobs[i];
      prof_begin(ctx, pex, ss);
      CKB(launch_energy_reduce(j.n_q, j.n_w, B[i].parts, B[i].w_q, B[i].zeta_w, B[i].eps, B[i].Ec, ss));
      prof_end(ctx, pex, ss, RPA_K_REDUCE, 1);
      ctx->launches++;
      char* r = pin + p.jobs[i].res_off;
      const size_t nqw = (size_t)j.n_q * j.n_w;
      CKB(cudaMemcpyAsync(r + 64, B[i].Ec, sizeof(double) * (3 * nqw + 1), cudaMemcpyDeviceToHost, ss));
      CKB(cudaMemcpyAsync(r, B[i].status, sizeof(int), cudaMemcpyDeviceToHost, ss));
      return RPA_OK;
    };
    for (size_t oi = 0; oi < order.size(); ++oi) {
      const int i = order[oi];
      cudaStream_t ss = bc.side[oi % nside];
      const rpa_job& j = jobs[i];
      if (j.prec == RPA_PREC_MIXED) {
        if (rpa_status st = stage_vside(ctx, pex, &j, B[i], 0, j.n_q, j.V, ss)) return st;
      } else {
        if (rpa_status st = stage_tail(ctx, pex, &j, B[i], 0, j.n_q, j.V, ss)) return st;
        if (rpa_status st = finish_job(i, ss)) return st;
      }
    }
    // join
    for (int k = 0; k < nside; ++k) {
      CKB(cudaEventRecord(bc.join[k], bc.side[k]));
      CKB(cudaStreamWaitEvent(s, bc.join[k], 0));
    }
    // ragged log-det of every (job, q, w) matrix of the mixed jobs, largest
    // matrices first (complex table, then real)
    if (g.n_task_c + g.n_task_r > 0) {
      std::vector<CholTask> tc, tr;
      for (int i = g.j0; i < g.j1; ++i) {
        const rpa_job& j = jobs[i];
        if (j.prec != RPA_PREC_MIXED) continue;
        const size_t es = j.is_complex ? 16 : 8;
        const size_t NN = (size_t)j.n_aux * j.n_aux * (es / 8);
        for (int q = 0; q < j.n_q; ++q)
          for (int w = 0; w < j.n_w; ++w) {
            const size_t b = (size_t)q * j.n_w + w;
            CholTask t{B[i].chi + b * NN, B[i].parts + 2 * b, B[i].L + q * NN, B[i].Vc + q * NN, B[i].ldV + q,
                       B[i].status, j.n_aux, 2, (int)(1 + b), 0};
            (j.is_complex ? tc : tr).push_back(t);
          }
      }
      auto by_size = [](const CholTask& a, const CholTask& c) { return a.N > c.N; };
      std::stable_sort(tc.begin(), tc.end(), by_size);
      std::stable_sort(tr.begin(), tr.end(), by_size);
      CholTask* hp = reinterpret_cast<CholTask*>(pin + g.pin_task);
      std::copy(tc.begin(), tc.end(), hp);
      std::copy(tr.begin(), tr.end(), hp + tc.size());
      CholTask* dp = reinterpret_cast<CholTask*>(ws + g.task_off);
      CKB(cudaMemcpyAsync(dp, hp, sizeof(CholTask) * (tc.size() + tr.size()), cudaMemcpyHostToDevice, s));
      prof_begin(ctx, pex, s);
      CKB(launch_cholesky_ragged(1, dp, (int)tc.size(), s));
      CKB(launch_cholesky_ragged(0, dp + tc.size(), (int)tr.size(), s));
      prof_end(ctx, pex, s, RPA_K_LOGDET, (tc.empty() ? 0 : 1) + (tr.empty() ? 0 : 1));
      ctx->launches += (tc.empty() ? 0 : 1) + (tr.empty() ? 0 : 1);
      for (int i = g.j0; i < g.j1; ++i)
        if (jobs[i].prec == RPA_PREC_MIXED)
          if (rpa_status st = finish_job(i, s)) return st;
    }
  }
  nk = ctx->launches.load() - l0;
  if (n_kernels) *n_kernels = nk;
  return RPA_OK;
}

}  // namespace rpa

using namespace rpa;

extern "C" rpa_status rpa_energy_batch(rpa_ctx* ctx, const rpa_job* jobs, int n_jobs, double* Ec_out) {
  if (!ctx || (!jobs && n_jobs > 0) || (!Ec_out && n_jobs > 0) || n_jobs < 0) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (n_jobs == 0) return RPA_OK;
  char msg[512];
  for (int i = 0; i < n_jobs; ++i) {
    if (validate_job(&jobs[i], msg, sizeof msg)) {
      ctx_set_error(ctx, "rpa_energy_batch: job %d: %s", i, msg);
      return RPA_E_INVAL;
    }
    if (jobs[i].mem != RPA_MEM_DEVICE) {
      ctx_set_error(ctx, "rpa_energy_batch: job %d is not device-resident", i);
      return RPA_E_INVAL;
    }
    if (jobs[i].ao) {
      ctx_set_error(ctx, "rpa_energy_batch: job %d is in AO form (run it with rpa_energy)", i);
      return RPA_E_INVAL;
    }
    if (jobs[i].prec == RPA_PREC_MIXED && !mixed_supported()) {
      ctx_set_error(ctx, "mixed-precision chi0 not supported by this library");
      return RPA_E_INVAL;
    }
  }
  CKB(cudaSetDevice(ctx->device));
  if (!ctx->batch) ctx->batch = new BatchCache;
  BatchCache& bc = *ctx->batch;
  if (!bc.side.init()) {
    ctx_set_error(ctx, "cannot create the batch side streams");
    return RPA_E_CUDA;
  }
  cudaStream_t s = ctx->ex.s;
  std::vector<uint64_t> sig = signature(jobs, n_jobs, ctx->n_slices);
  // with per-kernel profiling on, a known batch runs eagerly (a graph replay
  // cannot carry the timing marks)
  const bool known = bc.plan && bc.plan->exec && bc.plan->sig == sig;
  const bool replay = known && !ctx->prof;
  if (!known) {
    bc.plan = batch_plan(jobs, n_jobs, ctx->n_slices, ctx->cap);
    bc.plan->sig = sig;
  }
  Plan& p = *bc.plan;
  if (!bc.mem.ensure_ws(p.ws_bytes)) {
    ctx_set_error(ctx, "cannot allocate %zu bytes of batch workspace", p.ws_bytes);
    bc.plan.reset();
    return RPA_E_NOMEM;
  }
  if (!bc.pin.reserve(p.pin_bytes + 64)) {
    ctx_set_error(ctx, "cannot allocate pinned host staging");
    bc.plan.reset();
    return RPA_E_NOMEM;
  }
  char* pin = (char*)bc.pin.ptr;
  char* ws = (char*)bc.mem.ws;
  batch_fill_tables(p, jobs, n_jobs, pin);
  if (replay) {
    CKB(cudaGraphLaunch(p.exec, s));
    ctx->launches += p.kernels;
  } else {
    // eager run (the autotuner on for a new signature); results come from this run
    uint64_t nk = 0;
    if (rpa_status st = batch_enqueue(ctx, bc.side, p, jobs, ws, pin, s, !known, &nk, &ctx->ex)) {
      bc.plan.reset();
      return st;
    }
  }
  CKB(cudaEventRecord(ctx->ex.done, s));
  if (rpa_status st = wait_event(ctx, ctx->ex.done, ctx->timeout_s + p.work / 0.2e12)) return st;
  prof_collect(ctx, &ctx->ex);
  for (int i = 0; i < n_jobs; ++i) {
    const char* r = pin + p.jobs[i].res_off;
    int sw;
    memcpy(&sw, r, sizeof sw);
    if (rpa_status st = decode_status(ctx, sw, jobs[i].n_w)) {
      ctx_set_error(ctx, "rpa_energy_batch: job %d: %s", i, rpa_last_error(ctx));
      return st;
    }
    memcpy(&Ec_out[i], r + 64, sizeof(double));
  }
  if (!known) {
    // capture the same sequence (tuned plans now cached) for later calls
    cudaGraph_t graph = nullptr;
    CKB(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    uint64_t nk = 0;
    rpa_status st = batch_enqueue(ctx, bc.side, p, jobs, ws, pin, s, false, &nk, nullptr);
    ctx->launches -= nk;  // captured, not launched
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != RPA_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) {
      ctx_set_error(ctx, "batch graph capture failed: %s", cudaGetErrorString(ce));
      return RPA_E_CUDA;
    }
    ce = cudaGraphInstantiate(&p.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      p.exec = nullptr;
      ctx_set_error(ctx, "batch graph instantiation failed: %s", cudaGetErrorString(ce));
      return RPA_E_CUDA;
    }
    p.kernels = nk;
  }
  return RPA_OK;
}
