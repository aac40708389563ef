// Internal declarations shared by the librpa translation units (not part of
// the public C ABI in include/rpa.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/rpa.h"

namespace rpa {

// Devices whose attributes the library caches (ordinals at or above fall back
// to the entry of device 0).
constexpr int MAX_DEVICES = 64;
// Multiprocessor count of the current device, queried once per device.
int device_sm_count();

// Geometry of one q-batch handed to the kernels.  All pointers are device
// memory.  Matrices are row-major, complex data interleaved (re, im).
struct BatchGeom {
  int cplx;      // 1 complex128, 0 float64
  int n_aux;     // N
  int n_occ, n_virt, n_ov;
  int n_k;       // k-pairs per q
  int n_w;       // frequencies
  int n_qb;      // q-points in this batch
};

// ---- FP64 kernels (kernels_fp64.cu) --------------------------------------

// d[qb][j][w][t] = zeta_k * (-4 Delta / (Delta^2 + omega_w^2)),
// Delta = eps_virt[kq(qb,j)][a] - eps_occ[k(qb,j)][i], t = i*n_virt + a.
cudaError_t launch_dtab(const BatchGeom& g, const double* eps_occ, const double* eps_virt, const int* kidx,
                        const int* kqidx, const double* omega, double zeta_k, double* dtab, cudaStream_t s);

// chi[qb][w] (N x N, full Hermitian) = sum_j sum_t conj(C[qb*n_k+j][P,t]) C[..][Q,t] d[qb][j][w][t].
cudaError_t launch_chi0_fp64(const BatchGeom& g, const double* const* Cptrs, const double* dtab, double* chi,
                             cudaStream_t s);

// In-place Cholesky of n_mat matrices (stride bstride doubles).
//   mode 0: input Y = -Pi (lower triangle), factorises 1 + Y = 1 - Pi and writes
//           out[2*b] = ln det(1 - Pi) = sum log1p(pivot - 1), out[2*b+1] = Tr Pi.
//   mode 1: input V (lower triangle), writes the factor L (upper part zeroed);
//           out[b] = ln det V unless out is null.
//   mode 2: input chi of (q, w) = (b / n_w, b % n_w); factorises
//           M = V^-1 - chi with Wn[q] = -V^-1 (lower triangle) and writes
//           out[2*b] = ln det M + ldV[q] = ln det(1 - Pi), out[2*b+1] =
//           Tr(chi V) = Tr Pi, V read from Vc[q]; chi's strict upper triangle
//           is used as scratch (the input is read from the lower triangle).
// A non-positive pivot sets *status (if still 0) to 1 + status_base + b and
// the matrix is abandoned.
cudaError_t launch_cholesky(int cplx, int N, int n_mat, double* mats, long bstride, int mode, double* out,
                            int* status, int status_base, cudaStream_t s, const double* Wn = nullptr,
                            const double* Vc = nullptr, const double* ldV = nullptr, int n_w = 0);

// Kernel launches launch_cholesky makes for n_mat matrices of size N (1, or 2
// when a short last wave goes to clusters).
int cholesky_launches(int N, int n_mat);

// One matrix of a ragged Cholesky launch (matrices of different sizes).
struct CholTask {
  double* A;          // N x N, factorised in place
  double* out;        // mode 1: 1 double, modes 0 and 2: (ln det, Tr)
  const double* W;    // mode 2: -V^-1 of the matrix's q (lower triangle)
  const double* Vc;   // mode 2: V of the q
  const double* ldv;  // mode 2: ln det V of the q
  int* status;        // set to `code` on a non-positive pivot (if still 0)
  int N, mode, code, pad;
};
// Tasks in device memory, one CTA each; `cplx` selects complex128 or float64.
cudaError_t launch_cholesky_ragged(int cplx, const CholTask* tasks, int n_tasks, cudaStream_t s);

// Wn[q] = -V(q)^-1 (lower triangle) from the Cholesky factors L[q]: X = L^-1
// by block forward substitution into X[q], then -(X^H X).
cudaError_t launch_vinv(int cplx, int N, int n_q, const double* L, double* X, double* Wn, cudaStream_t s);

// ---- AO -> MO transform (kernels_ao.cu) -----------------------------------

// H[s][n] = sum_nu P[nu][s] c[nu][n0 + n], s < S, n < ncols: the half-
// transform of one k-point's PADF array P (n_bas x S) with the MO columns
// [n0, n0 + ncols) of c (n_bas x n_mo).  H is S x ncols.
cudaError_t launch_ao_half(int cplx, int n_bas, int S, int n_mo, const double* P, const double* c, int n0, int ncols,
                           double* H, cudaStream_t s);

// Lattice form of the PADF coefficients: n_R integer lattice vectors and the
// device arrays of their real cell-pair coefficients.
struct PadfLattice {
  static constexpr int kMax = 128;
  int n_R;
  int R[kMax][3];
  const double* C0[kMax];
};
// out[e] = sum_r C0[r][e] e^{2 pi i kfrac . R_r} for e < n (complex128 out),
// or the real part (cplx == 0, Gamma-equivalent k-points).
cudaError_t launch_padf_k(int cplx, const PadfLattice& L, const double* kfrac, long n, double* out, cudaStream_t s);

// Per (q, k) pair of one launch: MO coefficients at k and k+q, half-
// transforms H_occ(k) (S x n_occ) and H_virt(k+q) (S x n_virt), output
// C(q, k) (n_aux x n_occ*n_virt).
struct AoPairs {
  static constexpr int kMax = 48;
  const double* mo_k[kMax];
  const double* mo_kq[kMax];
  const double* h_occ[kMax];
  const double* h_virt[kMax];
  double* out[kMax];
};
// fit[gamma] = (first basis function of gamma's atom, basis functions on it,
// PADF column of (its first basis function, gamma), fit functions on it).
cudaError_t launch_ao_assemble(int cplx, const AoPairs& pr, int n_pairs, const int4* fit, int n_aux, int n_occ,
                               int n_virt, int n_mo, cudaStream_t s);

// ---- periodic projector (kernels_proj.cu) --------------------------------

// Per k-point (up to kMax): the overlap S (N x N, Hermitian positive
// definite), the MO coefficients c (N x n_mo) and the output c~ (may be c).
struct ProjPtrs {
  static constexpr int kMax = 256;
  const double* S[kMax];
  const double* c[kMax];
  double* out[kMax];
};
// W[k] (Np columns of N, column-major) = S(k) and V[k] = I; Np = N rounded
// up to even (a zero padding column).
cudaError_t launch_proj_load(int cplx, const ProjPtrs& P, int n_mat, int N, int Np, double* W, double* V,
                             cudaStream_t s);
// Round r of a one-sided Jacobi sweep over every W[k] (rotations accumulated
// in V[k]); pairs with |w_p^H w_q| / (|w_p| |w_q|) > thresh are rotated; the
// largest such ratio is merged into *off_max (the bits of a non-negative
// double).
cudaError_t launch_jacobi_round(int cplx, int n_mat, int N, int Np, int r, double* W, double* V, double thresh,
                                unsigned long long* off_max, cudaStream_t s);
// Eigenvalues (column norms of W) in ascending order into lam_sorted
// [n_mat][N], the column of each rank into by_rank, m = the largest count
// below eps_d over the k-points (into *m, zeroed by the caller), then
// out[k] = c[k] - U_m (U_m^H c[k]), U_m the columns of V of the m lowest
// ranks (X: scratch of n_mat * N * n_mo elements).
cudaError_t launch_proj_finish(int cplx, const ProjPtrs& P, int n_mat, int N, int Np, int n_mo, const double* W,
                               const double* V, double eps_d, double* lam_sorted, int* by_rank, int* m, double* X,
                               cudaStream_t s);

// T[b] = chi[b] * L[b / n_w]   (L lower triangular, N x N).
// Y[b] = -(L[b / n_w]^H T[b]), lower triangle only.
cudaError_t launch_sandwich(int cplx, int N, int n_batch, int n_w, const double* chi, const double* L, double* T,
                            double* Y, cudaStream_t s);

// Device-to-device copy by a kernel (a cudaMemcpyAsync when the pointers are
// not 16-byte aligned or the size is not a multiple of 16): for copies on a
// compute stream while the copy engines are busy with a job's host staging (a
// cudaMemcpyAsync there would wait behind those copies).
cudaError_t launch_copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s, uint64_t* n_launch = nullptr);

// E_c and the eps table from parts[q][w][2] = (ln det, Tr Pi):
// eps[q][w] = ln det + Tr, e_w = sum_q w_q eps[q][w], E = (1/2pi) sum_w zeta_w e_w.
cudaError_t launch_energy_reduce(int n_q, int n_w, const double* parts, const double* w_q, const double* zeta_w,
                                 double* eps, double* Ec, cudaStream_t s);

// Optional timing hook around groups of launches (cls: an RPA_K_* class).
struct LaunchHook {
  void* user;
  void (*begin)(void* user, cudaStream_t s);
  void (*end)(void* user, cudaStream_t s, int cls, int n_kernels);
};

// ---- mixed-precision kernels (kernels_mixed.cu) ----------------------------

// Bytes of mixed-path workspace for one q; slice_cap bounds the BF16 digit
// planes of the weighted operand (and so the frequencies per launch).
size_t mixed_workspace_bytes(const BatchGeom& g, int n_slices, size_t slice_cap);
// chi0 of one q for all frequencies on the tensor cores (split precision);
// `dtab` is the FP64 weight table of this q; a device time-out sets *status.
cudaError_t launch_chi0_mixed(const BatchGeom& g, int n_slices, const double* const* Cptrs, const double* dtab,
                              double* chi, void* work, size_t work_bytes, int* status, uint64_t* n_launch,
                              cudaStream_t s, size_t slice_cap, const LaunchHook* hook);
// One q of a multi-q mixed launch.
struct MixedQ {
  BatchGeom g;                 // n_qb = 1
  const double* const* Cptrs;  // device table of the q's n_k C blocks
  const double* dtab;          // device weights of the q, [n_k][n_w][n_ov]
  double* chi;                 // device output [n_w][N][N] (complex: interleaved)
  size_t slice_cap;            // 0: 12 GiB
};
// chi0 of n q-points, sharing persistent tensor-core launches (one per round
// of frequency groups).  tune: time the best split plans of each new shape
// class and record the fastest (must not be set under stream capture).
cudaError_t launch_chi0_mixed_multi(const MixedQ* qs, int n, int n_slices, void* work, size_t work_bytes,
                                    int* status, uint64_t* n_launch, cudaStream_t s, bool tune,
                                    const LaunchHook* hook = nullptr);
size_t mixed_multi_workspace_bytes(const MixedQ* qs, int n, int n_slices);
// chi0 of n q of one geometry one after another, the next q's weighted digit
// planes written by the tensor-core launch of the current one (two workspace
// regions, mixed_seq_workspace_bytes); otherwise one q at a time.
cudaError_t launch_chi0_mixed_seq(const MixedQ* qs, int n, int n_slices, void* work, size_t work_bytes,
                                  int* status, uint64_t* n_launch, cudaStream_t s, const LaunchHook* hook);
size_t mixed_seq_workspace_bytes(const BatchGeom& g, int n_slices, size_t slice_cap);
// ---- frequency-batched chi0 (freq_plan.cu) --------------------------------
// Transitions are split into windows (bins) of the transition energy D; in
// bin b the weight of every frequency node is a combination of the weights of
// rank[b] skeleton nodes, d(D, w) ~= sum_r coef[b][r][w] d(D, w_skel[b][r]),
// to FREQ_TOL of the bin's largest |d(., w)|.
constexpr int FREQ_MAX_BINS = 32;
constexpr double FREQ_TOL = 1e-10;
constexpr double FREQ_AMP = 16.0;
struct FreqPlan {
  int n_bins = 0;                         // 0: no plan (every frequency contracted)
  double edges[FREQ_MAX_BINS - 1] = {};   // interior edges, ascending: bin(D) = #{e : D >= e}
  int rank[FREQ_MAX_BINS] = {};
  double err[FREQ_MAX_BINS] = {};         // residual on the check grid / column maximum
  double amp[FREQ_MAX_BINS] = {};         // max over nodes of the scaled coefficient sum
  int rmax = 0;
  std::vector<int> skel;                  // [n_bins][rmax] node index (-1 unused)
  std::vector<double> coef;               // [n_bins][rmax][n_w]
  double work_ratio = 1.0;                // modelled sum_b rank K_b / (n_w K)
  double dlo = 0.0, dhi = 0.0;            // transition-energy window of the job
};
// Builds the plan from host copies of the band energies; mode 0 automatic
// (false when it saves no work), 1 off, 2 always.  Returns whether a plan is
// to be used.  With counts set it also returns every q's freq_counts for the
// plan ([q][n_k n_occ][n_bins], the input of freq_bin_q).
bool freq_plan_build(const rpa_job* j, const double* eps_occ_h, const double* eps_virt_h, int mode, FreqPlan* out,
                     std::vector<int>* counts = nullptr);
// fn(q) for q = 0..n_q-1 on up to 8 host threads (fn must not share state
// between q).
void freq_parallel_q(int n_q, const std::function<void(int)>& fn);
// cnt[(jj n_occ + i) n_bins + b]: virtual states of row (k-pair jj, occupied
// i) of q whose transition falls in bin b.  evs: virtual energies of every
// k-point sorted ascending.
void freq_counts(const rpa_job* j, const FreqPlan& p, int q, const double* eo, const double* evs, int* cnt);
int freq_bin_of(const FreqPlan& p, double D);

// One q of the frequency-batched chi0: positions of the bins (each padded to
// whole K-blocks) and the image of its device tables (pinned host memory):
//   ints:    row offsets [n_k n_occ][n_bins] | row counts [n_k n_occ][n_bins] |
//            parts [n_parts][3] (bin, first, end position; FREQ_PART at most) | rank [16]
//   doubles: skeleton frequencies [n_bins][rmax] | coef [n_bins][rmax][n_w] (shared by all q)
constexpr int FREQ_PART = 2048;
struct BinQHost {
  int Kt = 0, Kr = 0;  // positions, real K values (complex: 2 Kt)
  int tb0[FREQ_MAX_BINS + 1] = {};
  int n_parts = 0;
  const int* meta_i = nullptr;
  size_t n_meta_i = 0;
  const double* meta_d = nullptr;
  size_t n_meta_d = 0;
  // the same images already on the device (a job-wide copy made before any
  // other copy of the job is queued), or null: then each q's preparation
  // copies its image from the host
  const int* dmeta_i = nullptr;
  const double* dmeta_d = nullptr;
};
// Fills h (except the meta pointers) and the int image of q (from q's
// freq_counts when given, else counting here).
void freq_bin_q(const rpa_job* j, const FreqPlan& p, int q, const double* eo, const double* evs, BinQHost& h,
                std::vector<int>& img, const int* counts = nullptr);
// The double image shared by all q (skeleton frequencies, coefficients).
void freq_meta_d(const rpa_job* j, const FreqPlan& p, std::vector<double>& img);

// One q of a frequency-batched launch.
struct MixedBinQ {
  BatchGeom g;                 // n_qb = 1
  const double* const* Cptrs;  // device table of the q's n_k C blocks
  double* chi;                 // device output [n_w][N][N]
  const BinQHost* host;
  const double* eps_occ;       // device band energies and this q's pair indices
  const double* eps_virt;
  const int* kidx;
  const int* kqidx;
  double zeta_k;
  int* status;                 // device status word (plan mismatch)
};
// Workspace of the frequency-batched chi0 within `budget` bytes (pipelined
// with two q regions and two weighted-operand buffers when they fit); slots:
// skeleton slots per round, regions: 2 when pipelined, else 1.
size_t binned_workspace_bytes(const BatchGeom& g, const FreqPlan& p, int Kt_max, int n_parts_max, int n_slices,
                              size_t budget, int* slots = nullptr, int* regions = nullptr);
cudaError_t launch_chi0_binned(const MixedBinQ* qs, int n, const FreqPlan& p, int n_slices, void* work,
                               size_t work_bytes, int* status, uint64_t* n_launch, cudaStream_t s,
                               const LaunchHook* hook);
// Status word code of a device bin count that disagrees with the plan.
constexpr int STATUS_CODE_PLAN = 1 << 28;

// Autotuner cache (autotune.cu): the recorded split target for a shape-class
// key, 0 if none; autotune_record stores a measured choice.
int autotune_lookup(uint64_t key);
void autotune_record(uint64_t key, int value);
bool mixed_supported();
// Test hook: arm a dropped operand copy for the next tensor-core launch.
void mixed_test_drop_arm(int item);
int mixed_test_drop_take();
// Tensor-core flops the split-precision chi0 of one q executes (slice pairs
// x padded tiles x padded K).
uint64_t mixed_tensor_flops(const BatchGeom& g, int n_slices);
// Tensor-core flops issued by all split-precision chi0 launches of this process so far.
uint64_t mixed_tensor_flops_issued();

}  // namespace rpa
