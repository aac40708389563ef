// Periodic projector host side (proj.cu): workspace layout and the sweep loop.
#pragma once
#include <cuda_runtime.h>

#include "../../include/rpa.h"

struct rpa_ctx;

namespace rpa {

struct Exec;

// Offsets (bytes) of the projector's workspace: W and V (n_mat x Np x N),
// sorted eigenvalues, ranks, X (n_mat x N x n_mo), flags.
struct ProjLayout {
  int Np = 0;
  size_t W = 0, V = 0, lam = 0, rank = 0, X = 0, flags = 0, bytes = 0;
};
ProjLayout proj_layout(int cplx, int n_mat, int N, int n_mo);

// c~(k) = T(k) c(k) for n_mat k-points (out may equal c); synchronises s (a
// host test per Jacobi sweep).  *m_out: the number of removed eigen-
// directions; eig_host (optional, host [n_mat*N]): eigenvalues, ascending.
rpa_status run_projector(rpa_ctx* ctx, Exec* pex, int cplx, int n_mat, int N, int n_mo, const void* const* S,
                         const double* const* c, double* const* out, double eps_d, char* region, cudaStream_t s,
                         int* m_out, double* eig_host);

}  // namespace rpa
