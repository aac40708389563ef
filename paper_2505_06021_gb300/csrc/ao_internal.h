// AO-form jobs (rpa_job.ao): plan of the AO workspace region and the enqueue
// of the transform kernels (ao.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/rpa.h"

struct rpa_ctx;

namespace rpa {

struct Exec;

struct AoPlan {
  int S = 0, n_bas = 0;
  std::vector<int4> fit;                 // per fit function, see launch_ao_assemble
  std::vector<int> occ_slot, virt_slot;  // per k-point: H slot, -1 if unused
  int n_occ_slots = 0, n_virt_slots = 0;
  size_t occ_bytes = 0, virt_bytes = 0;  // one slot
  size_t cblk = 0;                       // one C(q, k_j) block
  size_t off_padf = 0, padf_bytes = 0;   // lattice form: one k-point's PADF array
  size_t off_proj = 0, off_cproj = 0, cproj_bytes = 0;  // projector: workspace, c~ per k-point
  size_t off_hocc = 0, off_hvirt = 0, off_c = 0, bytes = 0;
};

// RPA_OK or RPA_E_INVAL with a message; j->ao must be non-null.
int ao_validate(const rpa_job* j, char* msg, size_t len);
// qb: q whose MO-basis coefficients the region holds at once.
AoPlan ao_plan(const rpa_job* j, int qb);
// Bytes of the AO workspace region (0 for jobs without ao).
size_t ao_region_bytes(const rpa_job* j, int qb);
// Device bytes of the job's AO inputs (PADF and MO arrays of all k-points).
size_t ao_input_bytes(const rpa_job* j);
// Fit table upload and half-transforms of the k-points used by q (q < 0: by
// every q) into `region`.
rpa_status ao_enqueue_half(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const AoPlan& p, char* region, int q,
                           cudaStream_t s);
// With overlap matrices: the periodic projector's c~ of every k-point into the
// region (synchronises s); without: nothing.
rpa_status ao_project(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const AoPlan& p, char* region, cudaStream_t s);
// The MO coefficients the transform uses for k-point k (c~ or the job's c).
const double* ao_mo(const rpa_job* j, const AoPlan& p, const char* region, int k);
// C(q, k_j), j = 0..n_k-1, into out + j * cblk (half-transforms in place).
rpa_status ao_enqueue_assemble(rpa_ctx* ctx, Exec* pex, const rpa_job* j, const AoPlan& p, const char* region, int q,
                               char* out, cudaStream_t s);

}  // namespace rpa
