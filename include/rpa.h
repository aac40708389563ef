/*
 * librpa — GB300 (sm_103a) library for the hot path of the periodic RPA
 * correlation energy with density fitting and dual k-grids
 * (Spadetto, Philipsen, Foerster, Visscher, arXiv 2505.06021).
 *
 * For every q of the job's q-grid and every imaginary frequency omega the
 * library
 *   (A3) builds chi0_PQ(q, i omega) = zeta_k sum_k sum_{i in occ(k),
 *        a in virt(k+q)} conj(C_{P,ia}) C_{Q,ia} * (-4 Delta_ia /
 *        (Delta_ia^2 + omega^2)),  Delta_ia = eps_a(k+q) - eps_i(k)
 *        (Sec. 2.2, the fit-basis polarizability P^(0)_{gamma gamma'}; the
 *        resonant and complex-conjugate terms combined, occupations 2/0);
 *   (A4/A5) forms the symmetrised response Pi = V^(1/2) chi0 V^(1/2)
 *        (Sec. 2.1 working equation; Algorithm 1, "Z = V^0.5 P V^0.5");
 *   (A6) evaluates eps_{q,omega} = ln det(1 - Pi) + Tr Pi by an FP64
 *        Cholesky factorisation of 1 - Pi (Algorithm 1, the RPA integrand;
 *        sign as in eq. 1 of Sec. 2.1);
 *   (A7) reduces E_c = (1/2pi) sum_omega zeta_omega sum_q w_q eps_{q,omega}
 *        (Sec. 2.6, the (q, omega) double sum).
 *
 * Conventions
 * -----------
 * - Complex data is interleaved complex128 ((re, im) doubles); real data
 *   (Gamma-only jobs, is_complex = 0) is float64.  All matrices are
 *   row-major.  C(q, k_j) is n_aux x (n_occ*n_virt) with the pair index
 *   t = i*n_virt + a contiguous.  V(q) is n_aux x n_aux Hermitian positive
 *   definite (both triangles are read by the sandwich; only the lower one by
 *   the factorisation).
 * - Ownership: input buffers are borrowed; the caller keeps them alive and
 *   unmodified until the synchronous call returns, or, for rpa_submit, until
 *   rpa_poll / rpa_wait has reported completion.  Outputs go to caller
 *   buffers.  Device workspace belongs to the context.
 * - Errors: no exception crosses this boundary.  Every entry point returns an
 *   rpa_status; rpa_last_error() gives the message of the last failure on a
 *   context.  A non-positive pivot found on the device is reported as
 *   RPA_E_NOTPD (with q and omega in the message); kernels never trap.
 * - Streams: a `void *stream` argument is a cudaStream_t (0 = legacy default
 *   stream), e.g. torch.cuda.current_stream().cuda_stream.
 * - Determinism: in RPA_FP64 mode the same job gives bit-identical results
 *   whatever else runs on the device; all reductions have a fixed order.
 */
#ifndef RPA_H
#define RPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpa_ctx rpa_ctx;
typedef int rpa_status;

#define RPA_OK 0
#define RPA_E_INVAL 1    /* malformed job or argument */
#define RPA_E_NOMEM 2    /* device memory or admission cap exhausted */
#define RPA_E_CUDA 3     /* a CUDA runtime call failed */
#define RPA_E_NOTPD 4    /* V(q) or 1 - Pi(q, omega) not positive definite */
#define RPA_E_TIMEOUT 5  /* a bounded wait ran out */
#define RPA_E_BUSY 6     /* request queue full */
#define RPA_E_NOTREADY 7 /* submitted job not finished yet */

/* Arithmetic of the chi0 contraction.  The sandwich, the factorisation and
 * all sums are FP64 in every mode. */
#define RPA_PREC_FP64 0  /* chi0 in FP64 (DFMA) */
#define RPA_PREC_MIXED 1 /* chi0 on tcgen05 tensor cores from BF16 slices of
                            the FP64 operands, FP32 accumulation in exact
                            chunks, FP64 result (split-precision, Ozaki-style) */

/* Where a job's C, V and band-energy buffers live. */
#define RPA_MEM_DEVICE 0
#define RPA_MEM_HOST 1 /* host memory (pinned for speed): the library stages it
                          to device workspace per q, copies inside the call */

typedef struct {
  int device;           /* CUDA device ordinal */
  size_t hbm_cap_bytes; /* cap on workspace + admitted serving jobs; 0 = 120 GB */
  int n_slices;         /* BF16 slices per operand in RPA_PREC_MIXED (2..4; 0 = 4) */
  double timeout_s;     /* limit of every bounded wait (0 = 60 s) */
  int max_inflight;     /* serving: jobs admitted at once (0 = 64) */
  int chi0_freq;        /* RPA_PREC_MIXED chi0 of rpa_energy / rpa_chi0: 0 = frequency-batched when its
                           plan saves work (rpa_freq_plan), 1 = every frequency contracted, 2 = always
                           frequency-batched */
} rpa_config;

/* Atomic-orbital form of a job's fit coefficients (Sec. 2.2, PADF in
 * reciprocal space and the transformation to KS states).  Instead of the
 * MO-basis coefficients C(q, k_j) the job gives, per k-point kappa of K_G:
 *   - padf[kappa]: the k-dependent pair-atomic fit coefficients
 *     C_{nu mu alpha}(kappa), alpha a fit function on the atom of mu, as an
 *     n_bas x S matrix, S = sum_A n_bas_atom[A] n_fit_atom[A]: row nu, column
 *     sum_{A' < A} n_bas_atom[A'] n_fit_atom[A'] + (mu - first basis function
 *     of A) n_fit_atom[A] + (alpha - first fit function of A), A = atom(mu);
 *   - mo[kappa]: the KS (MO) coefficients c_{mu n}(kappa), n_bas x n_mo,
 *     occupied states in columns 0..n_occ-1, virtual states in columns
 *     n_occ..n_occ+n_virt-1.
 * Basis and fit functions are numbered atom by atom.  The library forms
 *   C_{gamma,ia}(q, k) = sum_{mu nu} conj(c_{mu i}(k)) c_{nu a}(k+q) B^{mu nu}_gamma,
 *   B^{mu nu}_gamma = [gamma on atom(mu)] C_{nu mu gamma}(k+q)
 *                   + [gamma on atom(nu)] conj(C_{mu nu gamma}(k)),
 * on the fly, one q at a time (k = k_j from pair_k, k+q from pair_kq), so the
 * MO-basis coefficients of the whole job never reside in memory at once.
 * Lattice form (n_R > 0, padf NULL): the job gives the real cell-pair
 * coefficients C^{0,dR} per lattice vector instead (same n_bas x S layout)
 * and the library forms each k-point's array as the lattice sum of Sec. 2.2,
 *   C_{nu mu alpha}(k) = sum_dR C^{0,dR}_{nu mu alpha} e^{i k . dR},
 * k . dR = 2 pi (kfrac . n), one k-point at a time in workspace.  Real
 * (Gamma-only) jobs need integer kfrac there.
 * Device memory only; the arrays are borrowed like C. */
typedef struct {
  int n_atoms;
  const int *n_bas_atom;   /* host [n_atoms]: basis functions per atom (> 0) */
  const int *n_fit_atom;   /* host [n_atoms]: fit functions per atom (> 0), sum = n_aux */
  int n_mo;                /* columns of every mo[kappa] (>= n_occ + n_virt, <= n_bas) */
  const void *const *padf; /* host [n_kpts] of device pointers, n_bas x S each (NULL: lattice form) */
  const void *const *mo;   /* host [n_kpts] of device pointers, n_bas x n_mo each */
  int n_R;                    /* lattice form: lattice vectors (1..128); 0 for the k form */
  const int *lattice;         /* host [n_R*3]: integer lattice vectors dR */
  const double *kfrac;        /* host [n_kpts*3]: fractional coordinates of the k-points */
  const void *const *padf_R;  /* host [n_R] of device pointers, real float64 n_bas x S each */
  const void *const *overlap; /* NULL, or host [n_kpts] of device pointers: the basis overlap S(kappa),
                                 n_bas x n_bas Hermitian positive definite; the MO coefficients are then
                                 regularised by the periodic projector (rpa_projector) first */
  double eps_d;               /* projector threshold on the eigenvalues of S(kappa) */
} rpa_ao;

typedef struct {
  int is_complex;                 /* 1: complex128 data; 0: real float64 (Gamma only) */
  int n_aux, n_occ, n_virt;       /* N, occupied and virtual bands per k */
  int n_q;                        /* q-points of the (dual) q-grid */
  int n_k;                        /* k-pairs per q (|K_reg|) */
  int n_w;                        /* imaginary frequencies */
  int n_kpts;                     /* rows of eps_occ / eps_virt (|K_G|) */
  const int *pair_k;              /* host [n_q*n_k]: row of eps_occ for k_j */
  const int *pair_kq;             /* host [n_q*n_k]: row of eps_virt for k_j+q */
  const double *w_q;              /* host [n_q]: q weights */
  double zeta_k;                  /* k weight (1/|K_reg|) */
  const double *omega;            /* host [n_w]: frequencies */
  const double *zeta_w;           /* host [n_w]: frequency weights */
  const double *eps_occ;          /* [n_kpts*n_occ], device or host (mem) */
  const double *eps_virt;         /* [n_kpts*n_virt], device or host (mem) */
  const void *const *C;           /* host array [n_q*n_k] of pointers to C(q,k_j); NULL with ao */
  const void *const *V;           /* host array [n_q] of pointers to V(q); with RPA_MEM_DEVICE every
                                     C and V pointer is aligned to its element size (16 bytes
                                     complex, 8 real), else RPA_E_INVAL */
  int prec;                       /* RPA_PREC_* */
  int mem;                        /* RPA_MEM_* */
  const rpa_ao *ao;               /* NULL, or the AO form of the fit coefficients (C must then be
                                     NULL and mem RPA_MEM_DEVICE; rpa_energy, rpa_chi0 and
                                     rpa_ao2mo take such jobs, the batch and serving calls do not) */
} rpa_job;

/* Create a context on cfg->device (NULL cfg = defaults).  Allocates nothing
 * large; workspace grows on first use.  RPA_E_CUDA if the device is absent. */
rpa_status rpa_create(const rpa_config *cfg, rpa_ctx **out);

/* Wait for outstanding work, free all workspace and the context. */
rpa_status rpa_destroy(rpa_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  Valid until the next call
 * on ctx.  With ctx == NULL: the last failure of rpa_create on this thread. */
const char *rpa_last_error(const rpa_ctx *ctx);

/* Host-only check of a job description (no device access; usable without a
 * GPU).  Writes a message into msg (if msg_len > 0) on failure. */
rpa_status rpa_job_validate(const rpa_job *job, char *msg, size_t msg_len);

/* Host-only: the frequency-batched form of the split-precision chi0 for this
 * job (job->mem must be RPA_MEM_HOST so that the band energies are readable
 * here; usable without a GPU).  chi0(w) of Sec. 2.2 weighs transition t by
 * d_t(w) = -4 D_t/(D_t^2 + w^2), a smooth function of its energy D_t, and
 * Algorithm 1 contracts once per frequency.  The library instead splits the
 * transitions of every q into n_bins windows of D (geometric, interior edges
 * edges[0..n_bins-2] ascending, D in bin b when exactly b edges are <= D) and
 * represents, inside bin b,
 *     d(D, omega_w) = sum_{r < rank[b]} coef[b][r][w] d(D, omega_{skel[b][r]})
 * (an interpolative decomposition over rank[b] of the job's own frequency
 * nodes, residual err[b] <= 1e-10 of the bin's largest |d(., omega_w)| on a
 * dense check grid), so chi0 needs rank[b] contractions over bin b instead of
 * n_w: chi0(w) = sum_b sum_r coef[b][r][w] X_{b,r}, X_{b,r} the contraction of
 * bin b's transitions at omega_{skel[b][r]}.  mode: 0 automatic (n_bins = 0
 * when the plan saves no work), 2 always.  Outputs (any may be NULL), with
 * B = RPA_FREQ_MAX_BINS: edges [B], rank [B], err [B], skel [B][n_w] (-1 past
 * rank[b]), coef [B][n_w][n_w] (row r of bin b), *work_ratio = modelled
 * sum_b rank[b] K_b / (n_w K).  RPA_E_INVAL for an invalid job or
 * mem != RPA_MEM_HOST. */
#define RPA_FREQ_MAX_BINS 32
rpa_status rpa_freq_plan(const rpa_job *job, int mode, int *n_bins, double *edges, int *rank, int *skel,
                         double *coef, double *err, double *work_ratio);

/* Host-only: device bytes the job occupies while it runs (its inputs when
 * mem == RPA_MEM_DEVICE plus the workspace of one q-batch) - the admission
 * footprint used by rpa_submit. */
rpa_status rpa_job_footprint(const rpa_job *job, size_t *bytes);

/* Step A3: chi0(q, i omega_w) for every w, written to the device buffer
 * chi_out [n_w][n_aux][n_aux] (full Hermitian matrices; complex128 or
 * float64).  Asynchronous on `stream`; job->mem must be RPA_MEM_DEVICE.  For
 * an AO-form job the coefficients of q are formed first, as by rpa_ao2mo. */
rpa_status rpa_chi0(rpa_ctx *ctx, const rpa_job *job, int q, void *chi_out, void *stream);

/* The AO -> MO transform of Sec. 2.2 for one q (job->ao must be set): writes
 * C(q, k_j) for j = 0..n_k-1 into the device buffer C_out [n_k][n_aux]
 * [n_occ*n_virt] (the layout of rpa_job.C).  FP64 throughout: each k-point's
 * PADF array is first contracted with its MO coefficients over its row index
 * (occupied columns for the k side, virtual ones for the k+q side), then each
 * pair sums over the basis functions on gamma's atom.  Asynchronous on
 * `stream`; intermediate arrays live in the context's workspace. */
rpa_status rpa_ao2mo(rpa_ctx *ctx, const rpa_job *job, int q, void *C_out, void *stream);

/* The periodic projector of Sec. 2.3 (job->ao with overlap): with
 * S(kappa) = U D U^H (eigenvalues ascending), R(kappa)_ii = Theta(D_ii - eps_d)
 * (Theta(0) = 1), R~ = prod_kappa R(kappa) over the job's k-points and
 * T(kappa) = U R~ U^H, writes c~(kappa) = T(kappa) c(kappa) into mo_out[kappa]
 * (host array [n_kpts] of device pointers, n_bas x n_mo each; may be the
 * job's own mo arrays).  Since the eigenvalues are ascending, R~ removes the
 * m lowest eigen-directions of every S(kappa), m = the largest count of
 * eigenvalues below eps_d; *n_removed (optional) receives m, eig_out
 * (optional, host [n_kpts*n_bas]) the eigenvalues.  Eigenvectors by a
 * one-sided Jacobi on the GPU (FP64); at most 256 k-points and
 * n_bas <= 6144.  Synchronises `stream` (one host test per Jacobi sweep);
 * RPA_E_TIMEOUT if 60 sweeps do not converge. */
rpa_status rpa_projector(rpa_ctx *ctx, const rpa_job *job, void *const *mo_out, double *eig_out, int *n_removed,
                         void *stream);

/* Steps A4-A6 for one q: from chi (device [n_w][n_aux][n_aux], as written by
 * rpa_chi0) computes out[2*w] = ln det(1 - Pi) and out[2*w+1] = Tr Pi,
 * Pi = V(q)^(1/2) chi V(q)^(1/2), into the HOST array out [n_w*2].
 * Synchronises `stream`.  RPA_E_NOTPD if V(q) or 1 - Pi is not positive
 * definite.  job->mem must be RPA_MEM_DEVICE. */
rpa_status rpa_logdet(rpa_ctx *ctx, const rpa_job *job, int q, const void *chi, double *out, void *stream);

/* The whole hot path A3-A7 for one job, synchronously on the context's own
 * stream: *Ec receives E_c; eps_qw (host [n_q*n_w] or NULL) the integrand
 * table eps_{q,w} = ln det + Tr; parts (host [n_q*n_w*2] or NULL) the pairs
 * (ln det(1 - Pi), Tr Pi).  Inputs on the device or, with mem ==
 * RPA_MEM_HOST, on the host (staged per q, copies overlapped with compute).
 * AO-form jobs (device memory): the half-transformed PADF arrays of every
 * k-point are formed once, then each q's MO-basis coefficients just before
 * its chi0. */
rpa_status rpa_energy(rpa_ctx *ctx, const rpa_job *job, double *Ec, double *eps_qw, double *parts);

/* Many independent jobs (uneven sizes) in one call: the split-precision
 * chi0 of every (job, q) shares persistent tensor-core launches (a segment
 * each), the jobs' tails run on side streams and their log-dets as one ragged
 * launch; the whole sequence is recorded once into a CUDA graph per batch
 * signature (shapes, precisions, device pointers) and replayed by later calls
 * with that signature (the first call runs eagerly and tunes the split-K
 * plans).  Ec_out (host [n_jobs]) receives each job's E_c.  Jobs must have
 * mem == RPA_MEM_DEVICE; the batch's workspace is cut into groups under the
 * context's HBM cap. */
rpa_status rpa_energy_batch(rpa_ctx *ctx, const rpa_job *jobs, int n_jobs, double *Ec_out);

/* Serving: enqueue a job (deep-copies the host descriptors; device buffers
 * stay borrowed).  The job is admitted once its footprint fits under the
 * context's cap next to the jobs already running; device-resident jobs that
 * wait together are admitted as one micro-batch whose (q, omega) work shares
 * the tensor-core launches, and up to four micro-batches share the device
 * (continuous batching).  RPA_E_BUSY if the queue is full, RPA_E_NOMEM if the
 * job alone exceeds the cap. */
rpa_status rpa_submit(rpa_ctx *ctx, const rpa_job *job, uint64_t *ticket);

/* RPA_E_NOTREADY until the ticket's job is done; then its status, with *Ec
 * and (optionally, host [n_q*n_w]) eps_qw filled.  A finished ticket can be
 * polled once; afterwards it is unknown (RPA_E_INVAL). */
rpa_status rpa_poll(rpa_ctx *ctx, uint64_t ticket, double *Ec, double *eps_qw);

/* rpa_poll with a bounded wait of at most timeout_s seconds
 * (RPA_E_TIMEOUT when it runs out). */
rpa_status rpa_wait(rpa_ctx *ctx, uint64_t ticket, double timeout_s, double *Ec, double *eps_qw);

/* Serving statistics since creation: jobs done, mean/p50/p99 latency from
 * submit to completion and p50/p99 queue wait, in seconds. */
rpa_status rpa_serving_stats(rpa_ctx *ctx, uint64_t *jobs_done, double *lat_mean, double *lat_p50,
                             double *lat_p99, double *wait_p50, double *wait_p99);

/* Serving high-water marks since creation: the most jobs running on the
 * device at once, the largest sum of their footprints (bytes) admitted under
 * the HBM cap, and the most jobs admitted together as one micro-batch (their
 * (q, omega) work shares launches).  Any pointer may be NULL. */
rpa_status rpa_serving_peak(rpa_ctx *ctx, int *max_running, size_t *max_bytes, int *max_batch);

/* Test hook for the failure path of the tensor-core chi0 kernel: the next
 * split-precision launch in this process leaves the operand copies of work
 * item `item` (and the producer's later ones) unissued, so the MMA thread's
 * bounded wait on that K-block runs out after its 2 s limit; the kernel raises
 * its error flag, drains, frees its tensor memory and returns, and the call
 * reports RPA_E_TIMEOUT.  The context stays usable.  No effect unless called. */
rpa_status rpa_test_drop_copy(rpa_ctx *ctx, int item);

/* Number of kernels this context has launched so far (all entry points). */
uint64_t rpa_kernel_launches(const rpa_ctx *ctx);

/* The context's own compute stream (a cudaStream_t) used by rpa_energy and
 * rpa_energy_batch; callers may record CUDA events on it. */
void *rpa_stream(rpa_ctx *ctx);

/* Per-kernel device timing (tracing).  rpa_profile(ctx, 1) resets and turns on
 * CUDA-event timing around every kernel the synchronous entry points launch
 * (events recorded on the launching stream); rpa_profile(ctx, 0) turns it off.
 * rpa_profile_read fills ms[RPA_K_COUNT] (summed device milliseconds) and
 * launches[RPA_K_COUNT] (kernel launches) per kernel class. */
#define RPA_K_DTAB 0     /* frequency-weight table */
#define RPA_K_CHI0 1     /* chi0 contraction kernel (FP64 or tensor-core) */
#define RPA_K_VFACTOR 2  /* Cholesky factor of V(q) */
#define RPA_K_SANDWICH 3 /* Pi = L^H chi0 L (two passes) */
#define RPA_K_LOGDET 4   /* Cholesky of 1 - Pi, ln det, Tr */
#define RPA_K_REDUCE 5   /* quadrature */
#define RPA_K_SLICE 6    /* operand preparation of the split-precision path */
#define RPA_K_CHI0_RED 7 /* split-K reduction of the tensor-core chi0 */
#define RPA_K_AO2MO 8    /* AO -> MO transform of the fit coefficients (AO-form jobs) */
#define RPA_K_PROJ 9     /* periodic projector (Jacobi sweeps, projection) */
#define RPA_K_H2D 10     /* host -> device staging copies of RPA_MEM_HOST jobs (copy stream; no kernels) */
#define RPA_K_COUNT 11
rpa_status rpa_profile(rpa_ctx *ctx, int enable);
rpa_status rpa_profile_read(rpa_ctx *ctx, double *ms, uint64_t *launches);

/* Work counters since the last rpa_profile(ctx, 1): *tensor_flops receives
 * the tensor-core flops issued by split-precision chi0 launches (slice pairs x
 * padded 128-row tiles x padded K, 2 flops per multiply-add; counted process
 * wide, so concurrent contexts add up), *h2d_bytes the bytes this context's
 * rpa_energy calls copied host -> device for RPA_MEM_HOST jobs.  Either
 * pointer may be NULL. */
rpa_status rpa_profile_counters(rpa_ctx *ctx, uint64_t *tensor_flops, uint64_t *h2d_bytes);

/* The log-det step (A4-A6) for callers that cannot allocate device memory at
 * call time - e.g. code embedded in a framework that owns all GPU memory
 * through its own pool, or latency-critical loops that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree.  The paper has no
 * counterpart; this is an interface convenience.
 *
 * Same results as rpa_logdet for one q, without a context: V (device,
 * n_aux x n_aux, Hermitian positive definite) and chi (device, n_w x n_aux x
 * n_aux, as written by rpa_chi0) are inputs; out (DEVICE, unlike rpa_logdet's
 * host array, n_w x 2 doubles) receives (ln det(1 - Pi), Tr Pi) per
 * frequency.  V, chi and out must be device (or managed) memory of the
 * current device, aligned to their element size (16 bytes complex, 8 real),
 * else RPA_E_INVAL; their sizes cannot be checked here, so the caller
 * guarantees n_aux^2, n_w n_aux^2 and 2 n_w elements.  Scratch is a fixed
 * static device array of 7,078,144 bytes that every GPU loading the library
 * holds until exit; nothing is allocated.  n_aux > 384 is rejected with
 * RPA_E_INVAL.  The first call on a device looks up the array's device
 * address (once per device, with that device current) and keeps it for the
 * life of the process, so do not reset the device (cudaDeviceReset) between
 * calls.  All calls share the array, so calls whose work overlaps on the GPU
 * (other streams or threads on the same device) race; serialise them.  The
 * call copies a status word to the host and synchronises `stream`, so it
 * cannot be made while that stream (or, in global capture mode, any stream)
 * is capturing.  Returns RPA_E_NOTPD / RPA_E_CUDA / RPA_E_INVAL with a message
 * in rpa_noalloc_last_error() (per host thread). */
rpa_status rpa_logdet_noalloc(int is_complex, int n_aux, int n_w, const void *V, const void *chi, double *out,
                              void *stream);
const char *rpa_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RPA_H */
