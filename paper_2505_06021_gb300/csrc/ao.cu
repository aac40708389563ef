// Host side of AO-form jobs (rpa_job.ao, Sec. 2.2): validation, the layout of
// the AO part of a lane's workspace, and the enqueue of the two transform
// kernels of kernels_ao.cu.
//
// Workspace region (offsets from Bufs.ao):
//   fit table   int4 per fit function gamma (see launch_ao_assemble)
//   PADF        lattice form only: one k-point's k-dependent PADF array
//   projector   with overlap matrices: the projector's workspace and the
//               regularised MO coefficients c~ of every k-point
//   H_occ       one S x n_occ slot per k-point that appears as k (pair_k)
//   H_virt      one S x n_virt slot per k-point that appears as k+q (pair_kq)
//   C           qb x n_k blocks n_aux x n_occ*n_virt: the MO-basis
//               coefficients of the q batch being processed (read by chi0)
// The half-transforms depend on the k-point only, so rpa_energy forms them
// once per job; each q then costs one assembly launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "ao_internal.h"
#include "proj_internal.h"
#include "rpa_internal.h"
#include "rpa_runtime.h"

namespace rpa {

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

int ao_validate(const rpa_job* j, char* msg, size_t len) {
  auto fail = [&](const char* m) {
    if (msg && len) snprintf(msg, len, "%s", m);
    return RPA_E_INVAL;
  };
  const rpa_ao* a = j->ao;
  if (j->C) return fail("AO-form job: C must be NULL (the coefficients are formed from ao)");
  if (j->mem != RPA_MEM_DEVICE) return fail("AO-form job: inputs must be in device memory");
  if (a->n_atoms <= 0 || !a->n_bas_atom || !a->n_fit_atom || !a->mo)
    return fail("AO-form job: n_atoms must be positive and the ao arrays non-NULL");
  if (a->n_R < 0 || a->n_R > PadfLattice::kMax)
    return fail("AO-form job: n_R must lie in [0, 128]");
  if (a->n_R > 0) {
    if (a->padf) return fail("AO-form job: give padf or the lattice form (n_R > 0), not both");
    if (!a->lattice || !a->kfrac || !a->padf_R) return fail("AO-form job: lattice form needs lattice, kfrac, padf_R");
    for (int r = 0; r < a->n_R; ++r)
      if (!a->padf_R[r]) return fail("AO-form job: a padf_R pointer is NULL");
    for (int k = 0; k < 3 * j->n_kpts; ++k) {
      if (!isfinite(a->kfrac[k])) return fail("AO-form job: kfrac not finite");
      if (!j->is_complex && a->kfrac[k] != floor(a->kfrac[k]))
        return fail("AO-form job: real (Gamma-only) lattice-form jobs need integer kfrac");
    }
  } else if (!a->padf) {
    return fail("AO-form job: padf is NULL and no lattice form given");
  }
  long nb = 0, nf = 0, S = 0;
  for (int A = 0; A < a->n_atoms; ++A) {
    if (a->n_bas_atom[A] <= 0 || a->n_fit_atom[A] <= 0)
      return fail("AO-form job: every atom needs at least one basis and one fit function");
    nb += a->n_bas_atom[A];
    nf += a->n_fit_atom[A];
    S += (long)a->n_bas_atom[A] * a->n_fit_atom[A];
  }
  if (nf != j->n_aux) return fail("AO-form job: fit functions per atom must sum to n_aux");
  if (a->overlap) {
    if (j->n_kpts > ProjPtrs::kMax) return fail("AO-form job: the projector takes at most 256 k-points");
    if (nb > 6144) return fail("AO-form job: the projector takes n_bas <= 6144");
    if (!isfinite(a->eps_d) || a->eps_d < 0.0) return fail("AO-form job: eps_d must be finite and >= 0");
    for (int k = 0; k < j->n_kpts; ++k)
      if (!a->overlap[k]) return fail("AO-form job: an overlap pointer is NULL");
  }
  if (a->n_mo < j->n_occ + j->n_virt || a->n_mo > nb)
    return fail("AO-form job: n_mo must lie in [n_occ + n_virt, n_bas]");
  if (nb > 65536 || S > (1L << 30)) return fail("AO-form job: basis or PADF array too large");
  for (int k = 0; k < j->n_kpts; ++k)
    if ((a->n_R == 0 && !a->padf[k]) || !a->mo[k]) return fail("AO-form job: a padf or mo pointer is NULL");
  return RPA_OK;
}

AoPlan ao_plan(const rpa_job* j, int qb) {
  AoPlan p;
  const rpa_ao* a = j->ao;
  const size_t es = j->is_complex ? 16 : 8;
  for (int A = 0; A < a->n_atoms; ++A) {
    p.n_bas += a->n_bas_atom[A];
    p.S += a->n_bas_atom[A] * a->n_fit_atom[A];
  }
  p.fit.resize(j->n_aux);
  for (int A = 0, b0 = 0, f0 = 0, s0 = 0; A < a->n_atoms; ++A) {
    const int nb = a->n_bas_atom[A], nf = a->n_fit_atom[A];
    for (int g = 0; g < nf; ++g) p.fit[f0 + g] = make_int4(b0, nb, s0 + g, nf);
    b0 += nb;
    f0 += nf;
    s0 += nb * nf;
  }
  p.occ_slot.assign(j->n_kpts, -1);
  p.virt_slot.assign(j->n_kpts, -1);
  for (long i = 0; i < (long)j->n_q * j->n_k; ++i) {
    if (p.occ_slot[j->pair_k[i]] < 0) p.occ_slot[j->pair_k[i]] = p.n_occ_slots++;
    if (p.virt_slot[j->pair_kq[i]] < 0) p.virt_slot[j->pair_kq[i]] = p.n_virt_slots++;
  }
  p.occ_bytes = al256(es * (size_t)p.S * j->n_occ);
  p.virt_bytes = al256(es * (size_t)p.S * j->n_virt);
  p.cblk = es * (size_t)j->n_aux * j->n_occ * j->n_virt;
  p.off_padf = al256(sizeof(int4) * (size_t)j->n_aux);
  p.padf_bytes = a->n_R > 0 ? al256(es * (size_t)p.n_bas * p.S) : 0;
  p.off_proj = p.off_padf + p.padf_bytes;
  size_t proj_bytes = 0;
  if (a->overlap) {
    proj_bytes = al256(proj_layout(j->is_complex, j->n_kpts, p.n_bas, a->n_mo).bytes);
    p.cproj_bytes = al256(es * (size_t)p.n_bas * a->n_mo);
  }
  p.off_cproj = p.off_proj + proj_bytes;
  p.off_hocc = p.off_cproj + p.cproj_bytes * (a->overlap ? j->n_kpts : 0);
  p.off_hvirt = p.off_hocc + p.occ_bytes * p.n_occ_slots;
  p.off_c = p.off_hvirt + p.virt_bytes * p.n_virt_slots;
  p.bytes = p.off_c + al256(p.cblk * j->n_k * (size_t)std::max(qb, 1));
  return p;
}

size_t ao_region_bytes(const rpa_job* j, int qb) { return j->ao ? ao_plan(j, qb).bytes : 0; }

size_t ao_input_bytes(const rpa_job* j) {
  if (!j->ao) return 0;
  const AoPlan p = ao_plan(j, 1);
  const size_t es = j->is_complex ? 16 : 8;
  if (j->ao->n_R > 0)
    return 8 * (size_t)j->ao->n_R * p.n_bas * p.S + es * (size_t)j->n_kpts * p.n_bas * j->ao->n_mo;
  return es * (size_t)j->n_kpts * p.n_bas * ((size_t)p.S + j->ao->n_mo);
}

#define CKA(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      ctx_set_error(ctx, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RPA_E_CUDA;                                                                             \
    }                                                                                                \
  } while (0)

const double* ao_mo(const rpa_job* j, const AoPlan& p, const char* region, int k) {
  if (j->ao->overlap) return (const double*)(region + p.off_cproj + p.cproj_bytes * (size_t)k);
  return (const double*)j->ao->mo[k];
}

rpa_status ao_project(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const AoPlan& p, char* region, cudaStream_t s) {
  const rpa_ao* a = j->ao;
  if (!a->overlap) return RPA_OK;
  std::vector<const double*> c(j->n_kpts);
  std::vector<double*> out(j->n_kpts);
  for (int k = 0; k < j->n_kpts; ++k) {
    c[k] = (const double*)a->mo[k];
    out[k] = (double*)(region + p.off_cproj + p.cproj_bytes * (size_t)k);
  }
  return run_projector(ctx, pex, j->is_complex, j->n_kpts, p.n_bas, a->n_mo, a->overlap, c.data(), out.data(),
                       a->eps_d, region + p.off_proj, s, nullptr, nullptr);
}

rpa_status ao_enqueue_half(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const AoPlan& p, char* region, int q,
                           cudaStream_t s) {
  const rpa_ao* a = j->ao;
  // the fit table (small, pageable source: consumed before the call returns)
  CKA(cudaMemcpyAsync(region, p.fit.data(), sizeof(int4) * p.fit.size(), cudaMemcpyHostToDevice, s));
  std::vector<char> need_o(j->n_kpts, 0), need_v(j->n_kpts, 0);
  const int q0 = q < 0 ? 0 : q, q1 = q < 0 ? j->n_q : q + 1;
  for (int qq = q0; qq < q1; ++qq)
    for (int jj = 0; jj < j->n_k; ++jj) {
      need_o[j->pair_k[(size_t)qq * j->n_k + jj]] = 1;
      need_v[j->pair_kq[(size_t)qq * j->n_k + jj]] = 1;
    }
  PadfLattice lat{};
  if (a->n_R > 0) {
    lat.n_R = a->n_R;
    for (int r = 0; r < a->n_R; ++r) {
      for (int d = 0; d < 3; ++d) lat.R[r][d] = a->lattice[3 * r + d];
      lat.C0[r] = (const double*)a->padf_R[r];
    }
  }
  int n = 0;
  prof_begin(ctx, pex, s);
  for (int k = 0; k < j->n_kpts; ++k) {
    if (!need_o[k] && !need_v[k]) continue;
    const double* P = (const double*)(a->n_R > 0 ? nullptr : a->padf[k]);
    if (a->n_R > 0) {  // this k-point's array as the lattice sum, into the PADF slot
      CKA(launch_padf_k(j->is_complex, lat, a->kfrac + 3 * k, (long)p.n_bas * p.S, (double*)(region + p.off_padf),
                        s));
      P = (const double*)(region + p.off_padf);
      ++n;
    }
    if (need_o[k]) {
      CKA(launch_ao_half(j->is_complex, p.n_bas, p.S, a->n_mo, P, ao_mo(j, p, region, k), 0, j->n_occ,
                         (double*)(region + p.off_hocc + p.occ_bytes * p.occ_slot[k]), s));
      ++n;
    }
    if (need_v[k]) {
      CKA(launch_ao_half(j->is_complex, p.n_bas, p.S, a->n_mo, P, ao_mo(j, p, region, k), j->n_occ, j->n_virt,
                         (double*)(region + p.off_hvirt + p.virt_bytes * p.virt_slot[k]), s));
      ++n;
    }
  }
  prof_end(ctx, pex, s, RPA_K_AO2MO, n);
  ctx->launches += n;
  return RPA_OK;
}

rpa_status ao_enqueue_assemble(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const AoPlan& p, const char* region, int q,
                               char* out, cudaStream_t s) {
  const rpa_ao* a = j->ao;
  int n = 0;
  prof_begin(ctx, pex, s);
  for (int j0 = 0; j0 < j->n_k; j0 += AoPairs::kMax) {
    const int np = std::min(AoPairs::kMax, j->n_k - j0);
    AoPairs pr{};
    for (int t = 0; t < np; ++t) {
      const size_t i = (size_t)q * j->n_k + j0 + t;
      const int k = j->pair_k[i], kq = j->pair_kq[i];
      pr.mo_k[t] = ao_mo(j, p, region, k);
      pr.mo_kq[t] = ao_mo(j, p, region, kq);
      pr.h_occ[t] = (const double*)(region + p.off_hocc + p.occ_bytes * p.occ_slot[k]);
      pr.h_virt[t] = (const double*)(region + p.off_hvirt + p.virt_bytes * p.virt_slot[kq]);
      pr.out[t] = (double*)(out + p.cblk * (size_t)(j0 + t));
    }
    CKA(launch_ao_assemble(j->is_complex, pr, np, (const int4*)region, j->n_aux, j->n_occ, j->n_virt, a->n_mo, s));
    ++n;
  }
  prof_end(ctx, pex, s, RPA_K_AO2MO, n);
  ctx->launches += n;
  return RPA_OK;
}

}  // namespace rpa
