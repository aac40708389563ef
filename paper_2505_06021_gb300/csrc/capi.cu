// C-ABI of librpa: context, job validation, workspace, and the orchestration
// of the RPA hot path (chi0 -> sandwich -> Cholesky log-det -> quadrature) on
// one GB300.  Declarations and argument contracts: include/rpa.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rpa_internal.h"
#include "ao_internal.h"
#include "rpa_runtime.h"

using namespace rpa;

static thread_local std::string g_create_error;

namespace rpa {

void ctx_set_error(rpa_ctx* ctx, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  std::lock_guard<std::mutex> g(ctx->err_mu);
  ctx->last_error = buf;
}

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      ctx_set_error(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RPA_E_CUDA;                                                                              \
    }                                                                                                 \
  } while (0)

// ------------------------------------------------------------------ Exec --

bool Exec::init() {
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return false;
  for (int i = 0; i < 2; ++i) {
    if (cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming) != cudaSuccess) return false;
  }
  if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) return false;
  return hres.reserve(4096);
}

void Exec::destroy() {
  if (s) cudaStreamSynchronize(s);
  if (cs) cudaStreamSynchronize(cs);
  if (ws) cudaFree(ws);
  ws = nullptr;
  ws_bytes = 0;
  if (s) cudaStreamDestroy(s);
  if (cs) cudaStreamDestroy(cs);
  for (int i = 0; i < 2; ++i) {
    if (ready[i]) cudaEventDestroy(ready[i]);
    if (freed[i]) cudaEventDestroy(freed[i]);
  }
  if (done) cudaEventDestroy(done);
  for (Mark& m : marks) {
    if (m.a) ev_pool.push_back(m.a);
    if (m.b) ev_pool.push_back(m.b);
  }
  marks.clear();
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  ev_pool.clear();
  s = cs = nullptr;
  done = nullptr;
  hstage.release();
  hbin.release();
  hres.release();
}

bool Exec::ensure_ws(size_t bytes) {
  if (ws_bytes >= bytes) return true;
  if (ws) {
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(cs);
    cudaFree(ws);
    ws = nullptr;
    ws_bytes = 0;
  }
  const size_t want = std::max(bytes, (size_t)64 << 20);
  if (cudaMalloc(&ws, want) != cudaSuccess) {
    cudaGetLastError();
    ws = nullptr;
    return false;
  }
  ws_bytes = want;
  return true;
}

rpa_status wait_event(rpa_ctx* ctx, cudaEvent_t ev, double timeout_s) {
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return RPA_OK;
    if (e != cudaErrorNotReady) {
      ctx_set_error(ctx, "device error: %s", cudaGetErrorString(e));
      return RPA_E_CUDA;
    }
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt > timeout_s) {
      ctx_set_error(ctx, "wait ran out after %.1f s", dt);
      return RPA_E_TIMEOUT;
    }
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(spins > 1000 ? 200 : 20));
  }
}

int device_sm_count() {
  static std::mutex mu;
  static int cache[MAX_DEVICES] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= MAX_DEVICES) dev = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 148;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

// ------------------------------------------------------------- tracing ----

cudaEvent_t Exec::take_event() {
  if (!ev_pool.empty()) {
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_begin(rpa_ctx* ctx, Exec* ex, cudaStream_t s) {
  if (!ctx->prof || !ex) return;
  Exec::Mark m{-1, 0, ex->take_event(), nullptr};
  if (m.a) cudaEventRecord(m.a, s);
  ex->marks.push_back(m);
}

void prof_end(rpa_ctx* ctx, Exec* ex, cudaStream_t s, int cls, int n_kernels) {
  if (!ctx->prof || !ex || ex->marks.empty()) return;
  Exec::Mark& m = ex->marks.back();
  m.cls = cls;
  m.n = n_kernels;
  m.b = ex->take_event();
  if (m.b) cudaEventRecord(m.b, s);
}

void prof_collect(rpa_ctx* ctx, Exec* ex) {
  if (!ex) return;
  for (Exec::Mark& m : ex->marks) {
    float ms = 0.f;
    if (m.a && m.b && m.cls >= 0 && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      ctx->prof_ms[m.cls] += ms;
      ctx->prof_n[m.cls] += m.n;
    }
    cudaGetLastError();
    if (m.a) ex->ev_pool.push_back(m.a);
    if (m.b) ex->ev_pool.push_back(m.b);
  }
  ex->marks.clear();
}

// ------------------------------------------------------------ validation --

static int set_msg(char* msg, size_t len, const char* fmt, ...) {
  if (msg && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, len, fmt, ap);
    va_end(ap);
  }
  return RPA_E_INVAL;
}

rpa_status validate_job(const rpa_job* j, char* msg, size_t len) {
  if (!j) return set_msg(msg, len, "job is NULL");
  if (j->is_complex != 0 && j->is_complex != 1) return set_msg(msg, len, "is_complex must be 0 or 1");
  if (j->n_aux <= 0 || j->n_occ <= 0 || j->n_virt <= 0)
    return set_msg(msg, len, "n_aux, n_occ, n_virt must be positive (got %d, %d, %d)", j->n_aux, j->n_occ,
                   j->n_virt);
  if (j->n_q <= 0 || j->n_k <= 0 || j->n_w <= 0 || j->n_kpts <= 0)
    return set_msg(msg, len, "n_q, n_k, n_w, n_kpts must be positive");
  if ((long long)j->n_occ * j->n_virt > (1LL << 28)) return set_msg(msg, len, "n_occ*n_virt too large");
  if (j->n_aux > 32768) return set_msg(msg, len, "n_aux > 32768 not supported");
  if ((long long)j->n_q * j->n_k > (1LL << 24)) return set_msg(msg, len, "n_q*n_k too large");
  if (!j->is_complex && (j->n_q != 1 || j->n_k != 1))
    return set_msg(msg, len, "real (is_complex=0) jobs are Gamma-only: n_q = n_k = 1");
  if (!j->pair_k || !j->pair_kq || !j->w_q || !j->omega || !j->zeta_w || !j->eps_occ || !j->eps_virt ||
      (!j->C && !j->ao) || !j->V)
    return set_msg(msg, len, "a required pointer is NULL");
  if (j->prec != RPA_PREC_FP64 && j->prec != RPA_PREC_MIXED) return set_msg(msg, len, "unknown prec %d", j->prec);
  if (j->prec == RPA_PREC_MIXED && j->n_w > 32)
    return set_msg(msg, len, "the split-precision path takes at most 32 frequencies (got %d)", j->n_w);
  if (j->mem != RPA_MEM_DEVICE && j->mem != RPA_MEM_HOST) return set_msg(msg, len, "unknown mem %d", j->mem);
  if (!(j->zeta_k > 0.0) || !isfinite(j->zeta_k)) return set_msg(msg, len, "zeta_k must be positive");
  for (long i = 0; i < (long)j->n_q * j->n_k; ++i) {
    if (j->pair_k[i] < 0 || j->pair_k[i] >= j->n_kpts || j->pair_kq[i] < 0 || j->pair_kq[i] >= j->n_kpts)
      return set_msg(msg, len, "pair index %ld out of range [0, %d)", i, j->n_kpts);
    if (!j->ao && !j->C[i]) return set_msg(msg, len, "C[%ld] is NULL", i);
    if (!j->ao && j->mem == RPA_MEM_DEVICE && ((uintptr_t)j->C[i] & (j->is_complex ? 15u : 7u)))
      return set_msg(msg, len, "C[%ld] is not aligned to its element size", i);
  }
  if (j->ao)
    if (int st = ao_validate(j, msg, len)) return st;
  for (int q = 0; q < j->n_q; ++q) {
    if (!j->V[q]) return set_msg(msg, len, "V[%d] is NULL", q);
    if (j->mem == RPA_MEM_DEVICE && ((uintptr_t)j->V[q] & (j->is_complex ? 15u : 7u)))
      return set_msg(msg, len, "V[%d] is not aligned to its element size", q);
    if (!isfinite(j->w_q[q])) return set_msg(msg, len, "w_q[%d] not finite", q);
  }
  for (int w = 0; w < j->n_w; ++w)
    if (!isfinite(j->omega[w]) || !isfinite(j->zeta_w[w]) || j->omega[w] < 0.0)
      return set_msg(msg, len, "omega/zeta_w[%d] invalid", w);
  return RPA_OK;
}

// -------------------------------------------------------------- layout ----

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace cap of the synchronous calls (the serving lanes use a smaller one).
size_t sync_ws_cap(rpa_ctx* ctx) { return std::min<size_t>(ctx->cap, (size_t)192 << 30); }

Layout plan_layout(const rpa_job* j, int qb, int n_slices, size_t ws_cap, bool mixed_ws, int qt, const BinJob* bj) {
  Layout L{};
  if (qt < qb) qt = qb;
  const size_t es = j->is_complex ? 16 : 8;
  const size_t NN = (size_t)j->n_aux * j->n_aux;
  const size_t nov = (size_t)j->n_occ * j->n_virt;
  const size_t npk = (size_t)j->n_q * j->n_k;
  const size_t nqw = (size_t)j->n_q * j->n_w;
  L.qb = qb;
  L.qt = qt;
  L.meta = al(sizeof(void*) * npk + sizeof(int) * 2 * npk + 64) +
           al(sizeof(double) * (2 * j->n_w + 2 * j->n_q + 3 * nqw + 8) + 64);
  L.dtab = al(sizeof(double) * qb * j->n_k * j->n_w * nov);
  L.chi = al(es * NN * qt * j->n_w);
  L.T = L.chi;
  L.L = al(es * NN * qt);
  if (j->mem == RPA_MEM_HOST) {
    L.stageC = al(es * j->n_aux * nov * qb * j->n_k);
    L.stageV = al(es * NN * qb);
    L.eps = al(sizeof(double) * (size_t)j->n_kpts * (j->n_occ + j->n_virt));
  }
  const bool binned = bj && bj->on && j->prec == RPA_PREC_MIXED;
  if (binned) L.dtab = 0;  // the frequency-batched chi0 forms its own weights
  if (j->prec == RPA_PREC_MIXED) {
    L.Vc = al(es * NN * qt);  // the inverse-form tail keeps a copy of V(q)
    if (mixed_ws && !binned) {
      BatchGeom g{j->is_complex, j->n_aux, j->n_occ, j->n_virt, (int)nov, j->n_k, j->n_w, 1};
      L.slice_cap = ws_cap / 2;
      L.mixed = al(mixed_workspace_bytes(g, n_slices, L.slice_cap));
    }
  }
  L.ao = al(ao_region_bytes(j, qb));
  if (binned) L.binmeta = al(bj->meta_bytes);
  L.total = L.meta + L.dtab + L.chi + L.T + L.L + L.Vc + 2 * (L.stageC + L.stageV) + L.eps + L.mixed + L.ao +
            L.binmeta;
  if (mixed_ws && binned) {
    // the frequency-batched chi0 takes what the cap leaves (pipelined when that suffices)
    BatchGeom g{j->is_complex, j->n_aux, j->n_occ, j->n_virt, (int)nov, j->n_k, j->n_w, 1};
    const size_t budget = ws_cap > L.total ? ws_cap - L.total : 0;
    L.mixed = al(binned_workspace_bytes(g, bj->plan, bj->Kt_max, bj->np_max, n_slices, budget));
    L.total += L.mixed;
  } else if (L.mixed && qb >= 2) {
    // two alternating regions (the next q's operand written during the
    // current q's tensor-core launch) when they fit under the cap
    BatchGeom g{j->is_complex, j->n_aux, j->n_occ, j->n_virt, (int)nov, j->n_k, j->n_w, 1};
    const size_t m2 = al(mixed_seq_workspace_bytes(g, n_slices, L.slice_cap));
    if (m2 > L.mixed && L.total - L.mixed + m2 <= ws_cap) {
      L.total += m2 - L.mixed;
      L.mixed = m2;
    }
  }
  return L;
}

int choose_qb(const rpa_job* j, int n_slices, size_t cap, const BinJob* bj) {
  int qb = j->n_q;
  if (j->ao) {  // AO form: the MO-basis coefficients of a few q at a time (<= 4 GB)
    const size_t per_q = (j->is_complex ? 16 : 8) * (size_t)j->n_aux * j->n_occ * j->n_virt * j->n_k;
    qb = (int)std::max<size_t>(1, std::min<size_t>((size_t)j->n_q, ((size_t)4 << 30) / std::max<size_t>(per_q, 1)));
  }
  while (qb > 1 && plan_layout(j, qb, n_slices, cap, true, 0, bj).total > cap) qb = (qb + 1) / 2;
  // host-resident inputs: at least four q-batches, so that the copies of one
  // batch overlap the compute of the previous one.  With the frequency-batched
  // chi0, fewer q per batch while that keeps all skeletons in one round (the
  // staging buffers and the chi0 workspace share the cap), and one q per batch
  // when its layout is not pipelined across q anyway: then every q is a launch
  // sequence of its own, and the only copy nothing overlaps, the first
  // batch's, is one q's.
  if (j->mem == RPA_MEM_HOST) {
    qb = std::min(qb, std::max(1, (j->n_q + 3) / 4));
    if (bj && bj->on && j->prec == RPA_PREC_MIXED) {
      auto layout = [&](int b, int& slots, int& regions) {
        const Layout L = plan_layout(j, b, n_slices, cap, false, j->n_q, nullptr);
        const size_t budget = cap > L.total ? cap - L.total : 0;
        const BatchGeom g{j->is_complex, j->n_aux, j->n_occ, j->n_virt, j->n_occ * j->n_virt, j->n_k, j->n_w, 1};
        binned_workspace_bytes(g, bj->plan, bj->Kt_max, bj->np_max, n_slices, budget, &slots, &regions);
      };
      int slots = 0, regions = 0;
      for (; qb > 1; --qb) {
        layout(qb, slots, regions);
        if (slots >= bj->plan.rmax) break;
      }
      if (qb > 1 && regions < 2) qb = 1;
    }
  }
  return qb;
}

int choose_qt(const rpa_job* j, int qb, int n_slices, size_t cap, const BinJob* bj) {
  // host-staged and AO-form jobs compute chi0 per staging batch; their tail
  // (V factor, log-det) runs over as many q as fit, so that its Cholesky
  // launches fill the GPU
  if (j->mem != RPA_MEM_HOST && !j->ao) return qb;
  int m = (j->n_q + qb - 1) / qb;
  while (m > 1 && plan_layout(j, qb, n_slices, cap, true, std::min(j->n_q, m * qb), bj).total > cap)
    m = (m + 1) / 2;
  return std::min(j->n_q, m * qb);
}

size_t job_workspace(const rpa_job* j, int n_slices, size_t ws_cap) {
  const int qb = choose_qb(j, n_slices, ws_cap);
  return plan_layout(j, qb, n_slices, ws_cap, true, choose_qt(j, qb, n_slices, ws_cap)).total;
}

size_t job_footprint(const rpa_job* j, int n_slices, size_t ws_cap) {
  const int qb = choose_qb(j, n_slices, ws_cap);
  Layout L = plan_layout(j, qb, n_slices, ws_cap, true, choose_qt(j, qb, n_slices, ws_cap));
  size_t in = 0;
  if (j->mem == RPA_MEM_DEVICE) {
    const size_t es = j->is_complex ? 16 : 8;
    in = j->ao ? ao_input_bytes(j) : es * (size_t)j->n_aux * j->n_occ * j->n_virt * j->n_q * j->n_k;
    in += es * (size_t)j->n_aux * j->n_aux * j->n_q;
  }
  return in + L.total;
}

Bufs carve(void* ws, const rpa_job* j, const Layout& L) {
  Bufs b{};
  const size_t npk = (size_t)j->n_q * j->n_k;
  const size_t nqw = (size_t)j->n_q * j->n_w;
  char* p = (char*)ws;
  char* m = p;
  b.Cptrs = (const void**)m;
  m += sizeof(void*) * npk;
  b.kidx = (int*)m;
  m += sizeof(int) * npk;
  b.kqidx = (int*)m;
  m = p + al(sizeof(void*) * npk + sizeof(int) * 2 * npk + 64);
  // doubles block, in the same order as the pinned upload/download images
  double* d = (double*)m;
  b.omega = d;
  d += j->n_w;
  b.zeta_w = d;
  d += j->n_w;
  b.w_q = d;
  d += j->n_q;
  b.Ec = d;
  d += 1;
  b.eps = d;
  d += nqw;
  b.parts = d;
  d += 2 * nqw;
  b.ldV = d;
  d += j->n_q;
  b.status = (int*)d;
  p += L.meta;
  b.dtab = (double*)p;
  p += L.dtab;
  b.chi = (double*)p;
  p += L.chi;
  b.T = (double*)p;
  p += L.T;
  b.L = (double*)p;
  p += L.L;
  b.Vc = L.Vc ? (double*)p : nullptr;
  p += L.Vc;
  for (int i = 0; i < 2; ++i) {
    b.stageC[i] = p;
    p += L.stageC;
    b.stageV[i] = p;
    p += L.stageV;
  }
  b.eps_occ = (double*)p;
  b.eps_virt = (double*)(p + sizeof(double) * (size_t)j->n_kpts * j->n_occ);
  p += L.eps;
  b.mixed = p;
  b.mixed_bytes = L.mixed;
  b.slice_cap = L.slice_cap;
  p += L.mixed;
  b.ao = L.ao ? p : nullptr;
  p += L.ao;
  b.binmeta = L.binmeta ? p : nullptr;
  return b;
}

size_t tables_bytes(const rpa_job* j) {
  const size_t npk = (size_t)j->n_q * j->n_k;
  const size_t tbytes = sizeof(void*) * npk + sizeof(int) * 2 * npk;
  return ((tbytes + 63) & ~(size_t)63) + sizeof(double) * (2 * j->n_w + j->n_q);
}

// Writes the job's small tables into pinned host memory `h` (tables_bytes of
// room): C pointers (device or staged), eps row indices, frequencies and
// weights.
void fill_tables_host(const rpa_job* j, const void* const* Cdev, char* h) {
  const size_t npk = (size_t)j->n_q * j->n_k;
  const size_t tbytes = sizeof(void*) * npk + sizeof(int) * 2 * npk;
  memcpy(h, Cdev, sizeof(void*) * npk);
  memcpy(h + sizeof(void*) * npk, j->pair_k, sizeof(int) * npk);
  memcpy(h + sizeof(void*) * npk + sizeof(int) * npk, j->pair_kq, sizeof(int) * npk);
  double* hd = (double*)(h + ((tbytes + 63) & ~(size_t)63));
  memcpy(hd, j->omega, sizeof(double) * j->n_w);
  memcpy(hd + j->n_w, j->zeta_w, sizeof(double) * j->n_w);
  memcpy(hd + 2 * j->n_w, j->w_q, sizeof(double) * j->n_q);
}

// Copies the tables at `h` to the device and zeroes the status word.  The
// copies read `h` when they execute, so a captured graph picks up whatever
// `h` holds at replay.
rpa_status enqueue_table_copies(rpa_ctx* ctx, const rpa_job* j, const Bufs& b, const char* h, cudaStream_t s) {
  const size_t npk = (size_t)j->n_q * j->n_k;
  const size_t tbytes = sizeof(void*) * npk + sizeof(int) * 2 * npk;
  const size_t dbytes = sizeof(double) * (2 * j->n_w + j->n_q);
  CK(cudaMemcpyAsync((void*)b.Cptrs, h, tbytes, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b.omega, h + ((tbytes + 63) & ~(size_t)63), dbytes, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(b.status, 0, sizeof(int), s));
  return RPA_OK;
}

static rpa_status upload_tables(rpa_ctx* ctx, Exec& ex, const rpa_job* j, const Bufs& b, const void* const* Cdev) {
  if (!ex.hstage.reserve(tables_bytes(j) + 64)) {
    ctx_set_error(ctx, "cannot allocate pinned host staging");
    return RPA_E_NOMEM;
  }
  fill_tables_host(j, Cdev, (char*)ex.hstage.ptr);
  return enqueue_table_copies(ctx, j, b, (const char*)ex.hstage.ptr, ex.s);
}

// d_t(omega) table for q in [q0, q0+nq).
rpa_status stage_dtab(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                      const double* eps_occ, const double* eps_virt, cudaStream_t s) {
  const int nk = j->n_k;
  BatchGeom g{j->is_complex, j->n_aux, j->n_occ, j->n_virt, j->n_occ * j->n_virt, nk, j->n_w, nq};
  prof_begin(ctx, pex, s);
  CK(launch_dtab(g, eps_occ, eps_virt, b.kidx + (size_t)q0 * nk, b.kqidx + (size_t)q0 * nk, b.omega, j->zeta_k,
                 b.dtab, s));
  prof_end(ctx, pex, s, RPA_K_DTAB, 1);
  ctx->launches++;
  return RPA_OK;
}

// The FP64 steps after chi0 for q in [q0, q0+nq), chi0 in b.chi: factor V,
// sandwich, Cholesky log-det.  V of the batch at Vdev[0..nq).
// V(q) of nq q-points into slots lo.. of L (and of the inverse form's copy Vc).
static rpa_status vside_copy(rpa_ctx* ctx, const rpa_job* j, const Bufs& b, int lo, int nq, const void* const* Vdev,
                             cudaStream_t s, bool staging = false) {
  const size_t es = j->is_complex ? 16 : 8;
  const size_t NN = (size_t)j->n_aux * j->n_aux;
  // with host staging, kernel copies: they run on the compute stream while the
  // copy engines are busy with the next batch's staging
  uint64_t nl = 0;
  for (int qi = 0; qi < nq; ++qi) {
    double* dst[2] = {b.L + (lo + qi) * NN * (es / 8), b.Vc ? b.Vc + (lo + qi) * NN * (es / 8) : nullptr};
    for (double* d : dst) {
      if (!d) continue;
      if (staging)
        CK(launch_copy_d2d(d, Vdev[qi], es * NN, s, &nl));
      else
        CK(cudaMemcpyAsync(d, Vdev[qi], es * NN, cudaMemcpyDeviceToDevice, s));
    }
  }
  ctx->launches += nl;
  return RPA_OK;
}

// V = L L^H for the q in [q0, q0+nq) held in slots 0..nq-1 of L (and, for the
// inverse form, ln det V and -V^-1 over L).
static rpa_status vside_factor(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                               cudaStream_t s) {
  const size_t es = j->is_complex ? 16 : 8;
  const size_t NN = (size_t)j->n_aux * j->n_aux;
  const long mstride = (long)(NN * (es / 8));
  prof_begin(ctx, pex, s);
  CK(launch_cholesky(j->is_complex, j->n_aux, nq, b.L, mstride, 1, b.Vc ? b.ldV + q0 : nullptr, b.status,
                     (1 << 29) + q0, s));
  prof_end(ctx, pex, s, RPA_K_VFACTOR, cholesky_launches(j->n_aux, nq));
  ctx->launches += cholesky_launches(j->n_aux, nq);
  if (b.Vc) {
    // inverse form: -V^-1 per q (X = L^-1 in T's storage, then -(X^H X) over L)
    prof_begin(ctx, pex, s);
    CK(launch_vinv(j->is_complex, j->n_aux, nq, b.L, b.T, b.L, s));
    prof_end(ctx, pex, s, RPA_K_VFACTOR, 2);
    ctx->launches += 2;
  }
  return RPA_OK;
}

rpa_status stage_vside(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                       const void* const* Vdev, cudaStream_t s) {
  if (rpa_status st = vside_copy(ctx, j, b, 0, nq, Vdev, s)) return st;
  return vside_factor(ctx, pex, j, b, q0, nq, s);
}

// Log-det of every (q, w), q in [q0, q0+nq) held in slots 0..nq-1 of chi, L
// and Vc (the V side done).
static rpa_status stage_logdet(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                               cudaStream_t s) {
  const size_t es = j->is_complex ? 16 : 8;
  const size_t NN = (size_t)j->n_aux * j->n_aux;
  const long mstride = (long)(NN * (es / 8));
  if (b.Vc) {
    // inverse form: one Cholesky of V^-1 - chi per (q, w); no sandwich
    prof_begin(ctx, pex, s);
    CK(launch_cholesky(j->is_complex, j->n_aux, nq * j->n_w, b.chi, mstride, 2, b.parts + (size_t)2 * q0 * j->n_w,
                       b.status, q0 * j->n_w, s, b.L, b.Vc, b.ldV + q0, j->n_w));
    prof_end(ctx, pex, s, RPA_K_LOGDET, cholesky_launches(j->n_aux, nq * j->n_w));
    ctx->launches += cholesky_launches(j->n_aux, nq * j->n_w);
    return RPA_OK;
  }
  // Y = -(L^H chi L) (lower triangle), overwriting chi's storage
  prof_begin(ctx, pex, s);
  CK(launch_sandwich(j->is_complex, j->n_aux, nq * j->n_w, j->n_w, b.chi, b.L, b.T, b.chi, s));
  prof_end(ctx, pex, s, RPA_K_SANDWICH, 2);
  ctx->launches += 2;
  // 1 - Pi' = 1 + Y: Cholesky, ln det, Tr
  prof_begin(ctx, pex, s);
  CK(launch_cholesky(j->is_complex, j->n_aux, nq * j->n_w, b.chi, mstride, 0, b.parts + (size_t)2 * q0 * j->n_w,
                     b.status, q0 * j->n_w, s));
  prof_end(ctx, pex, s, RPA_K_LOGDET, cholesky_launches(j->n_aux, nq * j->n_w));
  ctx->launches += cholesky_launches(j->n_aux, nq * j->n_w);
  return RPA_OK;
}

rpa_status stage_tail(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                      const void* const* Vdev, cudaStream_t s) {
  if (rpa_status st = stage_vside(ctx, pex, j, b, q0, nq, Vdev, s)) return st;
  return stage_logdet(ctx, pex, j, b, q0, nq, s);
}

// chi0 of q in [q0, q0+nq) into chi[0..nq) (device tables indexed by
// q*n_k + j; the d table of the batch is built first).
static rpa_status run_chi(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const Bufs& b, int q0, int nq,
                          const double* eps_occ, const double* eps_virt, cudaStream_t s, double* chi, int n_slices,
                          const BinJob* bj = nullptr) {
  const int nk = j->n_k;
  const size_t es = j->is_complex ? 16 : 8;
  const size_t NN = (size_t)j->n_aux * j->n_aux;
  BatchGeom g{j->is_complex, j->n_aux, j->n_occ, j->n_virt, j->n_occ * j->n_virt, nk, j->n_w, nq};
  if (j->prec == RPA_PREC_MIXED && bj && bj->on) {
    struct HookCtx {
      rpa_ctx* ctx;
      Exec* ex;
    } hc{ctx, pex};
    LaunchHook hook{&hc,
                    [](void* u, cudaStream_t st) {
                      HookCtx* h = (HookCtx*)u;
                      prof_begin(h->ctx, h->ex, st);
                    },
                    [](void* u, cudaStream_t st, int cls, int n) {
                      HookCtx* h = (HookCtx*)u;
                      prof_end(h->ctx, h->ex, st, cls, n);
                    }};
    BatchGeom g1 = g;
    g1.n_qb = 1;
    std::vector<MixedBinQ> mq(nq);
    for (int qi = 0; qi < nq; ++qi) {
      const int q = q0 + qi;
      mq[qi] = MixedBinQ{g1, (const double* const*)(b.Cptrs + (size_t)q * nk),
                         chi + (size_t)qi * j->n_w * NN * (es / 8),
                         &bj->qh[q], eps_occ, eps_virt, b.kidx + (size_t)q * nk, b.kqidx + (size_t)q * nk,
                         j->zeta_k, b.status};
    }
    uint64_t nl = 0;
    CK(launch_chi0_binned(mq.data(), nq, bj->plan, n_slices, b.mixed, b.mixed_bytes, b.status, &nl, s,
                          pex ? &hook : nullptr));
    ctx->launches += nl;
    return RPA_OK;
  }
  if (rpa_status st = stage_dtab(ctx, pex, j, b, q0, nq, eps_occ, eps_virt, s)) return st;
  if (j->prec == RPA_PREC_MIXED) {
    struct HookCtx {
      rpa_ctx* ctx;
      Exec* ex;
    } hc{ctx, pex};
    LaunchHook hook{&hc,
                    [](void* u, cudaStream_t st) {
                      HookCtx* h = (HookCtx*)u;
                      prof_begin(h->ctx, h->ex, st);
                    },
                    [](void* u, cudaStream_t st, int cls, int n) {
                      HookCtx* h = (HookCtx*)u;
                      prof_end(h->ctx, h->ex, st, cls, n);
                    }};
    BatchGeom g1 = g;
    g1.n_qb = 1;
    std::vector<MixedQ> mq(nq);
    for (int qi = 0; qi < nq; ++qi)
      mq[qi] = MixedQ{g1, (const double* const*)(b.Cptrs + (size_t)(q0 + qi) * nk),
                      b.dtab + (size_t)qi * nk * j->n_w * g.n_ov, chi + (size_t)qi * j->n_w * NN * (es / 8),
                      b.slice_cap};
    uint64_t nl = 0;
    CK(launch_chi0_mixed_seq(mq.data(), nq, n_slices, b.mixed, b.mixed_bytes, b.status, &nl, s,
                             pex ? &hook : nullptr));
    ctx->launches += nl;
  } else {
    prof_begin(ctx, pex, s);
    CK(launch_chi0_fp64(g, (const double* const*)(b.Cptrs + (size_t)q0 * nk), b.dtab, chi, s));
    prof_end(ctx, pex, s, RPA_K_CHI0, 1);
    ctx->launches++;
  }
  return RPA_OK;
}

rpa_status decode_status(rpa_ctx* ctx, int st, int n_w) {
  if (st == 0) return RPA_OK;
  const int code = st - 1;
  if (code == STATUS_CODE_PLAN) {
    ctx_set_error(ctx, "frequency-batched chi0: the device's transition counts disagree with the host plan");
    return RPA_E_CUDA;
  }
  if (code >= (1 << 30)) {
    ctx_set_error(ctx, "tensor-core chi0 kernel gave up waiting (code %d)", code - (1 << 30));
    return RPA_E_TIMEOUT;
  }
  if (code >= (1 << 29))
    ctx_set_error(ctx, "V(q=%d) is not positive definite", code - (1 << 29));
  else
    ctx_set_error(ctx, "1 - Pi(q=%d, w=%d) is not positive definite", code / n_w, code % n_w);
  return RPA_E_NOTPD;
}

rpa_status bin_job_build(rpa_ctx* ctx, Exec& ex, const rpa_job* j, BinJob& bj) {
  bj = BinJob{};
  if (j->prec != RPA_PREC_MIXED || ctx->chi0_freq == 1) return RPA_OK;
  const size_t no = (size_t)j->n_kpts * j->n_occ, nv = (size_t)j->n_kpts * j->n_virt;
  std::vector<double> eo, ev;
  const double* peo = j->eps_occ;
  const double* pev = j->eps_virt;
  if (j->mem == RPA_MEM_DEVICE) {
    eo.resize(no);
    ev.resize(nv);
    CK(cudaMemcpyAsync(eo.data(), j->eps_occ, sizeof(double) * no, cudaMemcpyDeviceToHost, ex.s));
    CK(cudaMemcpyAsync(ev.data(), j->eps_virt, sizeof(double) * nv, cudaMemcpyDeviceToHost, ex.s));
    CK(cudaStreamSynchronize(ex.s));
    peo = eo.data();
    pev = ev.data();
  }
  std::vector<int> counts;
  if (!freq_plan_build(j, peo, pev, ctx->chi0_freq, &bj.plan, &counts)) return RPA_OK;
  const size_t per_q = (size_t)j->n_k * j->n_occ * bj.plan.n_bins;
  std::vector<std::vector<int>> img(j->n_q);
  bj.qh.resize(j->n_q);
  freq_parallel_q(j->n_q,
                  [&](int q) { freq_bin_q(j, bj.plan, q, peo, nullptr, bj.qh[q], img[q], counts.data() + per_q * q); });
  size_t n_i = 0;
  for (int q = 0; q < j->n_q; ++q) {
    n_i += (img[q].size() + 15) & ~(size_t)15;
    bj.Kt_max = std::max(bj.Kt_max, bj.qh[q].Kt);
    bj.np_max = std::max(bj.np_max, bj.qh[q].n_parts);
  }
  std::vector<double> md;
  freq_meta_d(j, bj.plan, md);
  if (!ex.hbin.reserve(sizeof(int) * n_i + sizeof(double) * md.size() + 64)) {
    ctx_set_error(ctx, "cannot allocate pinned host staging");
    return RPA_E_NOMEM;
  }
  double* hd = (double*)ex.hbin.ptr;
  memcpy(hd, md.data(), sizeof(double) * md.size());
  int* hi = (int*)(hd + md.size());
  for (int q = 0; q < j->n_q; ++q) {
    memcpy(hi, img[q].data(), sizeof(int) * img[q].size());
    bj.qh[q].meta_i = hi;
    bj.qh[q].n_meta_i = img[q].size();
    bj.qh[q].meta_d = hd;
    bj.qh[q].n_meta_d = md.size();
    hi += (img[q].size() + 15) & ~(size_t)15;
  }
  bj.meta_bytes = (size_t)((char*)hi - (char*)ex.hbin.ptr);
  bj.on = true;
  return RPA_OK;
}

rpa_status energy_enqueue(rpa_ctx* ctx, Exec& ex, const rpa_job* job, size_t ws_cap, bool allow_bin) {
  char msg[512];
  if (validate_job(job, msg, sizeof msg)) {
    ctx_set_error(ctx, "%s", msg);
    return RPA_E_INVAL;
  }
  if (job->prec == RPA_PREC_MIXED && !mixed_supported()) {
    ctx_set_error(ctx, "mixed-precision chi0 not supported by this library");
    return RPA_E_INVAL;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ex.s;
  BinJob bj;
  if (allow_bin)
    if (rpa_status stb = bin_job_build(ctx, ex, job, bj)) return stb;
  const int qb = choose_qb(job, ctx->n_slices, ws_cap, &bj);
  const int qt = choose_qt(job, qb, ctx->n_slices, ws_cap, &bj);
  Layout L = plan_layout(job, qb, ctx->n_slices, ws_cap, true, qt, &bj);
  if (!ex.ensure_ws(L.total)) {
    ctx_set_error(ctx, "cannot allocate %zu bytes of workspace", L.total);
    return RPA_E_NOMEM;
  }
  Bufs b = carve(ex.ws, job, L);
  const size_t es = job->is_complex ? 16 : 8;
  const size_t NN = (size_t)job->n_aux * job->n_aux;
  const size_t nov = (size_t)job->n_occ * job->n_virt;
  const size_t cblk = es * job->n_aux * nov;
  const size_t nqw = (size_t)job->n_q * job->n_w;
  const bool host = job->mem == RPA_MEM_HOST;
  const int nbatch = (job->n_q + qb - 1) / qb;

  AoPlan aop;
  if (job->ao) aop = ao_plan(job, qb);
  std::vector<const void*> cp((size_t)job->n_q * job->n_k), vp(job->n_q);
  for (int q = 0; q < job->n_q; ++q) {
    const int bi = q / qb, slot = bi % 2, qi = q - bi * qb;
    for (int jj = 0; jj < job->n_k; ++jj) {
      const size_t i = (size_t)q * job->n_k + jj;
      if (job->ao)  // every batch's coefficients go to the same buffer
        cp[i] = b.ao + aop.off_c + ((size_t)qi * job->n_k + jj) * cblk;
      else
        cp[i] = host ? (const void*)(b.stageC[slot] + ((size_t)qi * job->n_k + jj) * cblk) : job->C[i];
    }
    vp[q] = host ? (const void*)(b.stageV[slot] + (size_t)qi * es * NN) : job->V[q];
  }
  if (rpa_status st0 = upload_tables(ctx, ex, job, b, cp.data())) return st0;
  if (b.binmeta) {
    // every q's bin tables in one copy, queued before the staging copies of
    // the inputs (a small copy behind those waits for the copy engine)
    CK(cudaMemcpyAsync(b.binmeta, ex.hbin.ptr, bj.meta_bytes, cudaMemcpyHostToDevice, s));
    for (int q = 0; q < job->n_q; ++q) {
      bj.qh[q].dmeta_i = (const int*)(b.binmeta + ((const char*)bj.qh[q].meta_i - (const char*)ex.hbin.ptr));
      bj.qh[q].dmeta_d = (const double*)(b.binmeta + ((const char*)bj.qh[q].meta_d - (const char*)ex.hbin.ptr));
    }
  }
  if (job->ao) {
    if (rpa_status st1 = ao_project(ctx, &ex, job, aop, b.ao, s)) return st1;
    if (rpa_status st1 = ao_enqueue_half(ctx, &ex, job, aop, b.ao, -1, s)) return st1;
  }

  const double* eo = job->eps_occ;
  const double* ev = job->eps_virt;
  // host staging: the copy stream fills stage[bi % 2] while the compute
  // stream works on the other slot
  auto issue_copy = [&](int bi) -> rpa_status {
    const int q0 = bi * qb, nq = std::min(qb, job->n_q - q0), slot = bi % 2;
    CK(cudaStreamWaitEvent(ex.cs, ex.freed[slot], 0));
    prof_begin(ctx, &ex, ex.cs);
    for (int i = 0; i < nq * job->n_k; ++i)
      CK(cudaMemcpyAsync(b.stageC[slot] + i * cblk, job->C[(size_t)q0 * job->n_k + i], cblk, cudaMemcpyHostToDevice,
                         ex.cs));
    for (int i = 0; i < nq; ++i)
      CK(cudaMemcpyAsync(b.stageV[slot] + i * es * NN, job->V[q0 + i], es * NN, cudaMemcpyHostToDevice, ex.cs));
    prof_end(ctx, &ex, ex.cs, RPA_K_H2D, 0);
    ctx->h2d_bytes += (uint64_t)nq * job->n_k * cblk + (uint64_t)nq * es * NN;
    CK(cudaEventRecord(ex.ready[slot], ex.cs));
    return RPA_OK;
  };
  if (host) {
    CK(cudaMemcpyAsync(b.eps_occ, job->eps_occ, sizeof(double) * job->n_kpts * job->n_occ, cudaMemcpyHostToDevice,
                       s));
    CK(cudaMemcpyAsync(b.eps_virt, job->eps_virt, sizeof(double) * job->n_kpts * job->n_virt,
                       cudaMemcpyHostToDevice, s));
    eo = b.eps_occ;
    ev = b.eps_virt;
    for (int i = 0; i < 2; ++i) CK(cudaEventRecord(ex.freed[i], s));
    for (int bi = 0; bi < std::min(2, nbatch); ++bi)
      if (rpa_status st = issue_copy(bi)) return st;
  }
  for (int bi = 0; bi < nbatch; ++bi) {
    const int q0 = bi * qb, nq = std::min(qb, job->n_q - q0), slot = bi % 2;
    const int t0 = (q0 / qt) * qt, lo = q0 - t0, nt = std::min(qt, job->n_q - t0);
    if (host) CK(cudaStreamWaitEvent(s, ex.ready[slot], 0));
    for (int qi = 0; job->ao && qi < nq; ++qi)
      if (rpa_status st1 = ao_enqueue_assemble(ctx, &ex, job, aop, b.ao, q0 + qi,
                                               b.ao + aop.off_c + (size_t)qi * job->n_k * cblk, s))
        return st1;
    if (rpa_status st = run_chi(ctx, &ex, job, b, q0, nq, eo, ev, s, b.chi + (size_t)lo * job->n_w * NN * (es / 8),
                                ctx->n_slices, &bj))
      return st;
    if (rpa_status st = vside_copy(ctx, job, b, lo, nq, vp.data() + q0, s, host)) return st;
    // the tail once its batch of q is complete (chi, V of every q in place)
    if (q0 + nq == t0 + nt) {
      if (rpa_status st = vside_factor(ctx, &ex, job, b, t0, nt, s)) return st;
      if (rpa_status st = stage_logdet(ctx, &ex, job, b, t0, nt, s)) return st;
    }
    if (host) {
      CK(cudaEventRecord(ex.freed[slot], s));
      if (bi + 2 < nbatch)
        if (rpa_status st2 = issue_copy(bi + 2)) return st2;
    }
  }
  prof_begin(ctx, &ex, s);
  CK(launch_energy_reduce(job->n_q, job->n_w, b.parts, b.w_q, b.zeta_w, b.eps, b.Ec, s));
  prof_end(ctx, &ex, s, RPA_K_REDUCE, 1);
  ctx->launches++;
  if (!ex.hres.reserve(64 + sizeof(double) * (3 * nqw + 1))) {
    ctx_set_error(ctx, "cannot allocate pinned result buffer");
    return RPA_E_NOMEM;
  }
  CK(cudaMemcpyAsync(ex.results(), b.Ec, sizeof(double) * (3 * nqw + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&ex.status_word(), b.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ex.done, s));
  return RPA_OK;
}

rpa_status energy_finish(rpa_ctx* ctx, Exec& ex, const rpa_job* job, double* Ec, double* eps_qw, double* parts) {
  const size_t nqw = (size_t)job->n_q * job->n_w;
  prof_collect(ctx, &ex);
  if (rpa_status st = decode_status(ctx, ex.status_word(), job->n_w)) return st;
  const double* r = ex.results();
  if (Ec) *Ec = r[0];
  if (eps_qw) memcpy(eps_qw, r + 1, sizeof(double) * nqw);
  if (parts) memcpy(parts, r + 1 + nqw, sizeof(double) * 2 * nqw);
  return RPA_OK;
}


}  // namespace rpa

// ============================================================== C ABI =====

extern "C" {

rpa_status rpa_create(const rpa_config* cfg, rpa_ctx** out) {
  if (!out) return RPA_E_INVAL;
  *out = nullptr;
  rpa_config c{};
  if (cfg) c = *cfg;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return RPA_E_CUDA;
  }
  if (c.device < 0 || c.device >= n) {
    g_create_error = "device ordinal out of range";
    return RPA_E_INVAL;
  }
  if (c.n_slices == 0) c.n_slices = 4;
  if (c.n_slices < 2 || c.n_slices > 4) {
    g_create_error = "n_slices must be in [2, 4]";
    return RPA_E_INVAL;
  }
  rpa_ctx* ctx = new rpa_ctx();
  ctx->device = c.device;
  ctx->n_slices = c.n_slices;
  ctx->cap = c.hbm_cap_bytes ? c.hbm_cap_bytes : (size_t)120 << 30;
  ctx->timeout_s = c.timeout_s > 0 ? c.timeout_s : 60.0;
  ctx->max_inflight = c.max_inflight > 0 ? c.max_inflight : 64;
  if (c.chi0_freq < 0 || c.chi0_freq > 2) {
    g_create_error = "chi0_freq must be 0, 1 or 2";
    delete ctx;
    return RPA_E_INVAL;
  }
  ctx->chi0_freq = c.chi0_freq;
  if (cudaSetDevice(c.device) != cudaSuccess || !ctx->ex.init()) {
    g_create_error = std::string("stream/event creation failed: ") + cudaGetErrorString(cudaGetLastError());
    ctx->ex.destroy();
    delete ctx;
    return RPA_E_CUDA;
  }
  *out = ctx;
  return RPA_OK;
}

rpa_status rpa_destroy(rpa_ctx* ctx) {
  if (!ctx) return RPA_E_INVAL;
  rpa::serving_shutdown(ctx);
  cudaSetDevice(ctx->device);
  rpa::batch_release(ctx);
  ctx->ex.destroy();
  delete ctx;
  return RPA_OK;
}

const char* rpa_last_error(const rpa_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->last_error.c_str();
}

rpa_status rpa_job_validate(const rpa_job* job, char* msg, size_t msg_len) {
  if (msg && msg_len) msg[0] = 0;
  return validate_job(job, msg, msg_len);
}

rpa_status rpa_job_footprint(const rpa_job* job, size_t* bytes) {
  if (!bytes) return RPA_E_INVAL;
  if (rpa_status st = validate_job(job, nullptr, 0)) return st;
  *bytes = job_footprint(job, 4, (size_t)24 << 30);
  return RPA_OK;
}

uint64_t rpa_kernel_launches(const rpa_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

void* rpa_stream(rpa_ctx* ctx) { return ctx ? (void*)ctx->ex.s : nullptr; }

rpa_status rpa_profile(rpa_ctx* ctx, int enable) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->prof = enable != 0;
  for (int i = 0; i < RPA_K_COUNT; ++i) {
    ctx->prof_ms[i] = 0.0;
    ctx->prof_n[i] = 0;
  }
  if (ctx->prof) {
    ctx->flops0 = mixed_tensor_flops_issued();
    ctx->h2d_bytes = 0;
  }
  return RPA_OK;
}

rpa_status rpa_profile_counters(rpa_ctx* ctx, uint64_t* tensor_flops, uint64_t* h2d_bytes) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (tensor_flops) *tensor_flops = mixed_tensor_flops_issued() - ctx->flops0;
  if (h2d_bytes) *h2d_bytes = ctx->h2d_bytes.load();
  return RPA_OK;
}

rpa_status rpa_profile_read(rpa_ctx* ctx, double* ms, uint64_t* launches) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (int i = 0; i < RPA_K_COUNT; ++i) {
    if (ms) ms[i] = ctx->prof_ms[i];
    if (launches) launches[i] = ctx->prof_n[i];
  }
  return RPA_OK;
}

rpa_status rpa_chi0(rpa_ctx* ctx, const rpa_job* job, int q, void* chi_out, void* stream) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  char msg[512];
  if (validate_job(job, msg, sizeof msg)) {
    ctx_set_error(ctx, "%s", msg);
    return RPA_E_INVAL;
  }
  if (q < 0 || q >= job->n_q || !chi_out) {
    ctx_set_error(ctx, "rpa_chi0: q out of range or chi_out NULL");
    return RPA_E_INVAL;
  }
  if (job->mem != RPA_MEM_DEVICE) {
    ctx_set_error(ctx, "rpa_chi0 needs device-resident inputs (mem = RPA_MEM_DEVICE)");
    return RPA_E_INVAL;
  }
  if (job->prec == RPA_PREC_MIXED && !mixed_supported()) {
    ctx_set_error(ctx, "mixed-precision chi0 not supported by this library");
    return RPA_E_INVAL;
  }
  CK(cudaSetDevice(ctx->device));
  Exec& ex = ctx->ex;
  cudaStream_t s = (cudaStream_t)stream;
  BinJob bj;
  if (rpa_status stb = bin_job_build(ctx, ex, job, bj)) return stb;
  Layout L = plan_layout(job, 1, ctx->n_slices, sync_ws_cap(ctx), true, 0, &bj);
  if (!ex.ensure_ws(L.total)) {
    ctx_set_error(ctx, "cannot allocate %zu bytes of workspace", L.total);
    return RPA_E_NOMEM;
  }
  Bufs b = carve(ex.ws, job, L);
  std::vector<const void*> cp;
  AoPlan aop;
  if (job->ao) {
    aop = ao_plan(job, 1);
    cp.resize((size_t)job->n_q * job->n_k);
    for (size_t i = 0; i < cp.size(); ++i) cp[i] = b.ao + aop.off_c + (i % job->n_k) * aop.cblk;
  }
  // the lane's uploads run on ex.s; order the caller's stream after them
  if (rpa_status st0 = upload_tables(ctx, ex, job, b, job->ao ? cp.data() : job->C)) return st0;
  CK(cudaEventRecord(ex.done, ex.s));
  CK(cudaStreamWaitEvent(s, ex.done, 0));
  if (job->ao) {
    if (rpa_status st1 = ao_project(ctx, &ex, job, aop, b.ao, s)) return st1;
    if (rpa_status st1 = ao_enqueue_half(ctx, &ex, job, aop, b.ao, q, s)) return st1;
    if (rpa_status st1 = ao_enqueue_assemble(ctx, &ex, job, aop, b.ao, q, b.ao + aop.off_c, s)) return st1;
  }
  if (rpa_status st = run_chi(ctx, &ex, job, b, q, 1, job->eps_occ, job->eps_virt, s, (double*)chi_out,
                              ctx->n_slices, &bj))
    return st;
  // the d table in the workspace is reused by the next call on this context
  CK(cudaEventRecord(ex.done, s));
  rpa_status wst = wait_event(ctx, ex.done, ctx->timeout_s + 600.0);
  prof_collect(ctx, &ex);
  if (wst) return wst;
  int stw = 0;
  CK(cudaMemcpy(&stw, b.status, sizeof(int), cudaMemcpyDeviceToHost));
  return decode_status(ctx, stw, job->n_w);
}

rpa_status rpa_ao2mo(rpa_ctx* ctx, const rpa_job* job, int q, void* C_out, void* stream) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  char msg[512];
  if (validate_job(job, msg, sizeof msg)) {
    ctx_set_error(ctx, "%s", msg);
    return RPA_E_INVAL;
  }
  if (!job->ao || q < 0 || q >= job->n_q || !C_out) {
    ctx_set_error(ctx, "rpa_ao2mo: job without ao, q out of range or C_out NULL");
    return RPA_E_INVAL;
  }
  CK(cudaSetDevice(ctx->device));
  Exec& ex = ctx->ex;
  cudaStream_t s = (cudaStream_t)stream;
  const AoPlan aop = ao_plan(job, 1);
  // only the AO region is used: fit table and half-transforms
  if (!ex.ensure_ws(aop.off_c + 256)) {
    ctx_set_error(ctx, "cannot allocate %zu bytes of workspace", aop.off_c);
    return RPA_E_NOMEM;
  }
  char* region = (char*)ex.ws;
  if (rpa_status st = ao_project(ctx, &ex, job, aop, region, s)) return st;
  if (rpa_status st = ao_enqueue_half(ctx, &ex, job, aop, region, q, s)) return st;
  if (rpa_status st = ao_enqueue_assemble(ctx, &ex, job, aop, region, q, (char*)C_out, s)) return st;
  // the workspace is reused by the next call on this context
  CK(cudaEventRecord(ex.done, s));
  rpa_status wst = wait_event(ctx, ex.done, ctx->timeout_s + 600.0);
  prof_collect(ctx, &ex);
  return wst;
}

rpa_status rpa_logdet(rpa_ctx* ctx, const rpa_job* job, int q, const void* chi, double* out, void* stream) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  char msg[512];
  if (validate_job(job, msg, sizeof msg)) {
    ctx_set_error(ctx, "%s", msg);
    return RPA_E_INVAL;
  }
  if (q < 0 || q >= job->n_q || !chi || !out || job->mem != RPA_MEM_DEVICE) {
    ctx_set_error(ctx, "rpa_logdet: bad q, NULL pointer or host-resident job");
    return RPA_E_INVAL;
  }
  CK(cudaSetDevice(ctx->device));
  Exec& ex = ctx->ex;
  cudaStream_t s = (cudaStream_t)stream;
  rpa_job j1 = *job;
  j1.prec = RPA_PREC_FP64;
  Layout L = plan_layout(&j1, 1, ctx->n_slices, sync_ws_cap(ctx), true);
  if (!ex.ensure_ws(L.total)) {
    ctx_set_error(ctx, "cannot allocate %zu bytes of workspace", L.total);
    return RPA_E_NOMEM;
  }
  Bufs b = carve(ex.ws, &j1, L);
  const size_t es = job->is_complex ? 16 : 8;
  const size_t NN = (size_t)job->n_aux * job->n_aux;
  CK(cudaMemsetAsync(b.status, 0, sizeof(int), s));
  CK(cudaMemcpyAsync(b.L, job->V[q], es * NN, cudaMemcpyDeviceToDevice, s));
  prof_begin(ctx, &ex, s);
  CK(launch_cholesky(job->is_complex, job->n_aux, 1, b.L, (long)(NN * (es / 8)), 1, nullptr, b.status,
                     (1 << 29) + q, s));
  prof_end(ctx, &ex, s, RPA_K_VFACTOR, 1);
  prof_begin(ctx, &ex, s);
  CK(launch_sandwich(job->is_complex, job->n_aux, job->n_w, job->n_w, (const double*)chi, b.L, b.T, b.chi, s));
  prof_end(ctx, &ex, s, RPA_K_SANDWICH, 2);
  prof_begin(ctx, &ex, s);
  CK(launch_cholesky(job->is_complex, job->n_aux, job->n_w, b.chi, (long)(NN * (es / 8)), 0, b.parts, b.status, 0,
                     s));
  prof_end(ctx, &ex, s, RPA_K_LOGDET, 1);
  ctx->launches += 4;
  if (!ex.hres.reserve(64 + sizeof(double) * 2 * job->n_w)) return RPA_E_NOMEM;
  CK(cudaMemcpyAsync(ex.results(), b.parts, sizeof(double) * 2 * job->n_w, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&ex.status_word(), b.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ex.done, s));
  if (rpa_status st = wait_event(ctx, ex.done, ctx->timeout_s + 600.0)) return st;
  prof_collect(ctx, &ex);
  const int sw = ex.status_word();
  if (sw) {
    const int code = sw - 1;
    if (code >= (1 << 29))
      ctx_set_error(ctx, "V(q=%d) is not positive definite", q);
    else
      ctx_set_error(ctx, "1 - Pi(q=%d, w=%d) is not positive definite", q, code);
    return RPA_E_NOTPD;
  }
  memcpy(out, ex.results(), sizeof(double) * 2 * job->n_w);
  return RPA_OK;
}

rpa_status rpa_test_drop_copy(rpa_ctx* ctx, int item) {
  if (!ctx || item < 0) return RPA_E_INVAL;
  mixed_test_drop_arm(item);
  return RPA_OK;
}

rpa_status rpa_energy(rpa_ctx* ctx, const rpa_job* job, double* Ec, double* eps_qw, double* parts) {
  if (!ctx || !Ec) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (rpa_status st = rpa::energy_enqueue(ctx, ctx->ex, job, rpa::sync_ws_cap(ctx), true)) return st;
  // bounded wait: scaled with the job's chi0 work at a conservative 0.2 TFLOP/s
  const double work = 8.0 * job->n_aux * (double)job->n_aux * job->n_occ * job->n_virt * job->n_q * job->n_k *
                      job->n_w / (job->is_complex ? 1.0 : 4.0);
  const double limit = ctx->timeout_s + work / 0.2e12;
  if (rpa_status st = rpa::wait_event(ctx, ctx->ex.done, limit)) return st;
  return rpa::energy_finish(ctx, ctx->ex, job, Ec, eps_qw, parts);
}

}  // extern "C"
