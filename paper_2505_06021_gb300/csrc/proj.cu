// Host side of the periodic projector (Sec. 2.3): the Jacobi sweep loop with
// its convergence test, the rpa_projector entry point, and the regularised MO
// coefficients of AO-form jobs that carry overlap matrices.
#include <cuda_runtime.h>
#include <float.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "proj_internal.h"
#include "rpa_internal.h"
#include "rpa_runtime.h"

namespace rpa {

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int kMaxSweeps = 60;
}  // namespace

ProjLayout proj_layout(int cplx, int n_mat, int N, int n_mo) {
  ProjLayout L;
  const size_t es = cplx ? 16 : 8;
  L.Np = N + (N & 1);
  L.W = 0;
  L.V = L.W + al256(es * (size_t)n_mat * L.Np * N);
  L.lam = L.V + al256(es * (size_t)n_mat * L.Np * N);
  L.rank = L.lam + al256(sizeof(double) * (size_t)n_mat * N);
  L.X = L.rank + al256(sizeof(int) * (size_t)n_mat * N);
  L.flags = L.X + al256(es * (size_t)n_mat * N * n_mo);
  L.bytes = L.flags + 256;
  return L;
}

rpa_status run_projector(rpa_ctx* ctx, Exec* pex, int cplx, int n_mat, int N, int n_mo, const void* const* S,
                         const double* const* c, double* const* out, double eps_d, char* region, cudaStream_t s,
                         int* m_out, double* eig_host) {
  if (n_mat > ProjPtrs::kMax) {
    ctx_set_error(ctx, "projector: at most %d k-points", ProjPtrs::kMax);
    return RPA_E_INVAL;
  }
  const ProjLayout L = proj_layout(cplx, n_mat, N, n_mo);
  ProjPtrs P{};
  for (int k = 0; k < n_mat; ++k) {
    P.S[k] = (const double*)S[k];
    P.c[k] = c[k];
    P.out[k] = out[k];
  }
  double* W = (double*)(region + L.W);
  double* V = (double*)(region + L.V);
  unsigned long long* off = (unsigned long long*)(region + L.flags);
  int* m = (int*)(region + L.flags + 64);
  auto fail = [&](cudaError_t e, const char* what) {
    ctx_set_error(ctx, "projector: %s failed: %s", what, cudaGetErrorString(e));
    return RPA_E_CUDA;
  };
  cudaError_t e = launch_proj_load(cplx, P, n_mat, N, L.Np, W, V, s);
  if (e != cudaSuccess) return fail(e, "load");
  ctx->launches += 1;
  // rotate pairs above the rounding level of a length-N inner product; stop
  // once no pair of a sweep is further from orthogonal than a few times that
  const double rot_thresh = 1e-15;
  const double conv = std::max(1e-14, 4.0 * N * DBL_EPSILON);
  int sweep = 0;
  double off_h = 1.0;
  prof_begin(ctx, pex, s);
  for (; sweep < kMaxSweeps && off_h > conv; ++sweep) {
    if ((e = cudaMemsetAsync(off, 0, sizeof(unsigned long long), s)) != cudaSuccess) return fail(e, "memset");
    for (int r = 0; r < L.Np - 1; ++r)
      if ((e = launch_jacobi_round(cplx, n_mat, N, L.Np, r, W, V, rot_thresh, off, s)) != cudaSuccess)
        return fail(e, "Jacobi round");
    ctx->launches += L.Np - 1;
    unsigned long long bits = 0;
    if ((e = cudaMemcpyAsync(&bits, off, sizeof bits, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return fail(e, "copy");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "sync");
    memcpy(&off_h, &bits, sizeof off_h);
  }
  prof_end(ctx, pex, s, RPA_K_PROJ, sweep * (L.Np - 1));
  if (off_h > conv) {
    ctx_set_error(ctx, "projector: Jacobi not converged after %d sweeps (off-orthogonality %.3g)", kMaxSweeps, off_h);
    return RPA_E_TIMEOUT;
  }
  if ((e = cudaMemsetAsync(m, 0, sizeof(int), s)) != cudaSuccess) return fail(e, "memset");
  if ((e = cudaMemsetAsync(region + L.rank, 0xff, sizeof(int) * (size_t)n_mat * N, s)) != cudaSuccess)
    return fail(e, "memset");
  prof_begin(ctx, pex, s);
  e = launch_proj_finish(cplx, P, n_mat, N, L.Np, n_mo, W, V, eps_d, (double*)(region + L.lam),
                         (int*)(region + L.rank), m, (double*)(region + L.X), s);
  if (e != cudaSuccess) return fail(e, "finish");
  prof_end(ctx, pex, s, RPA_K_PROJ, 3);
  ctx->launches += 3;
  int mh = 0;
  if ((e = cudaMemcpyAsync(&mh, m, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(e, "copy");
  if (eig_host && (e = cudaMemcpyAsync(eig_host, region + L.lam, sizeof(double) * (size_t)n_mat * N,
                                       cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return fail(e, "copy");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "sync");
  if (m_out) *m_out = mh;
  return RPA_OK;
}

}  // namespace rpa

using namespace rpa;

extern "C" rpa_status rpa_projector(rpa_ctx* ctx, const rpa_job* job, void* const* mo_out, double* eig_out,
                                    int* n_removed, void* stream) {
  if (!ctx) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  char msg[512];
  if (validate_job(job, msg, sizeof msg)) {
    ctx_set_error(ctx, "%s", msg);
    return RPA_E_INVAL;
  }
  if (!job->ao || !job->ao->overlap || !mo_out) {
    ctx_set_error(ctx, "rpa_projector: needs an AO-form job with overlap matrices and mo_out");
    return RPA_E_INVAL;
  }
  for (int k = 0; k < job->n_kpts; ++k)
    if (!mo_out[k]) {
      ctx_set_error(ctx, "rpa_projector: mo_out[%d] is NULL", k);
      return RPA_E_INVAL;
    }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    ctx_set_error(ctx, "cudaSetDevice failed");
    return RPA_E_CUDA;
  }
  const rpa_ao* a = job->ao;
  int n_bas = 0;
  for (int A = 0; A < a->n_atoms; ++A) n_bas += a->n_bas_atom[A];
  const ProjLayout L = proj_layout(job->is_complex, job->n_kpts, n_bas, a->n_mo);
  Exec& ex = ctx->ex;
  if (!ex.ensure_ws(L.bytes)) {
    ctx_set_error(ctx, "cannot allocate %zu bytes of workspace", L.bytes);
    return RPA_E_NOMEM;
  }
  std::vector<const double*> c(job->n_kpts);
  std::vector<double*> out(job->n_kpts);
  for (int k = 0; k < job->n_kpts; ++k) {
    c[k] = (const double*)a->mo[k];
    out[k] = (double*)mo_out[k];
  }
  rpa_status st = run_projector(ctx, &ex, job->is_complex, job->n_kpts, n_bas, a->n_mo, a->overlap, c.data(),
                                out.data(), a->eps_d, (char*)ex.ws, (cudaStream_t)stream, n_removed, eig_out);
  prof_collect(ctx, &ex);
  return st;
}
