/*
 * Plain FP64 CPU oracle for the periodic RPA correlation-energy hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * reads this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or table with the GPU
 * path.
 *
 * Every routine is the textbook definition written out with plain loops in
 * double precision and compensated (Neumaier) summation for long sums.  No
 * blocking, fusion or reordering beyond what the definitions state.
 *
 * Paper: Spadetto, Philipsen, Foerster, Visscher, "Periodic implementation of
 * the random phase approximation with numerical atomic orbitals and dual
 * reciprocal space grids" (arXiv 2505.06021).
 *
 * Complex matrices are stored interleaved (re, im) row-major; real matrices
 * are plain row-major doubles.  All pointers are host memory.
 *
 * Return codes: 0 ok, 1 invalid argument, 4 matrix not positive definite,
 * 5 Jacobi did not converge.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- sums -- */

typedef struct {
  double s, c;
} nsum_t;

static inline void nsum_add(nsum_t *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nsum_get(const nsum_t *a) { return a->s + a->c; }

static inline double re_(const double *m, int is_c, size_t i) { return is_c ? m[2 * i] : m[i]; }
static inline double im_(const double *m, int is_c, size_t i) { return is_c ? m[2 * i + 1] : 0.0; }

/* ------------------------------------------------------- response chi0 -- */
/*
 * Density-fitted independent-particle response at one q and one imaginary
 * frequency omega (Sec. 2.2, the fit-basis polarizability P^(0)_{gamma
 * gamma'}(q, i omega), with occupations 2/0, spin compensation, and the
 * resonant plus complex-conjugate term combined):
 *
 *   chi_PQ = zeta_k sum_j sum_{i,a} conj(C_j[P,ia]) C_j[Q,ia] d_ia,
 *   d_ia   = -4 Delta_ia / (Delta_ia^2 + omega^2),
 *   Delta_ia = eps_virt_j[a] - eps_occ_j[i],
 *
 * j running over the n_k pairs (k_j, k_j + q) of this q; eps_occ_j are the
 * occupied energies at k_j and eps_virt_j the virtual ones at k_j + q.
 * C_j is n_aux x (n_occ*n_virt), pair index t = i*n_virt + a.
 * Every (P, Q) entry is summed independently (Hermiticity is not assumed).
 * chi_out: n_aux x n_aux.
 */
int oracle_chi0(int is_complex, int n_aux, int n_occ, int n_virt, int n_k, const double *const *C,
                const double *const *eps_occ, const double *const *eps_virt, double zeta_k, double omega,
                double *chi_out, int n_threads) {
  if (n_aux <= 0 || n_occ <= 0 || n_virt <= 0 || n_k <= 0) return 1;
  const int n_ov = n_occ * n_virt;
  double *d = (double *)malloc(sizeof(double) * (size_t)n_k * n_ov);
  if (!d) return 1;
  for (int j = 0; j < n_k; ++j)
    for (int i = 0; i < n_occ; ++i)
      for (int a = 0; a < n_virt; ++a) {
        double delta = eps_virt[j][a] - eps_occ[j][i];
        d[(size_t)j * n_ov + (size_t)i * n_virt + a] = -4.0 * delta / (delta * delta + omega * omega);
      }
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int P = 0; P < n_aux; ++P) {
    for (int Q = 0; Q < n_aux; ++Q) {
      nsum_t sr = {0, 0}, si = {0, 0};
      for (int j = 0; j < n_k; ++j) {
        const double *Cj = C[j];
        for (int t = 0; t < n_ov; ++t) {
          size_t ip = (size_t)P * n_ov + t, iq = (size_t)Q * n_ov + t;
          double ar = re_(Cj, is_complex, ip), ai = im_(Cj, is_complex, ip);
          double br = re_(Cj, is_complex, iq), bi = im_(Cj, is_complex, iq);
          double w = d[(size_t)j * n_ov + t];
          /* conj(a) * b = (ar br + ai bi) + i (ar bi - ai br) */
          nsum_add(&sr, (ar * br + ai * bi) * w);
          if (is_complex) nsum_add(&si, (ar * bi - ai * br) * w);
        }
      }
      size_t o = (size_t)P * n_aux + Q;
      if (is_complex) {
        chi_out[2 * o] = zeta_k * nsum_get(&sr);
        chi_out[2 * o + 1] = zeta_k * nsum_get(&si);
      } else {
        chi_out[o] = zeta_k * nsum_get(&sr);
      }
    }
  }
  free(d);
  return 0;
}

/* ------------------------------------- k-dependent PADF coefficients -- */
/*
 * The k-dependent pair-atomic fit coefficients of one k-point from the
 * cell-pair coefficients (Sec. 2.2, the lattice sum defining C(k)):
 *   C_{nu mu alpha}(k) = sum_{dR} C^{0,dR}_{nu mu alpha} e^{i k . dR},
 * with k . dR = 2 pi (kappa . n) for the fractional coordinates kappa of k
 * and the integer lattice vector n of dR.  C0[r] (n_entries real values)
 * holds the coefficients of lattice vector R[3r..3r+2]; out receives
 * n_entries complex values (re, im).  One compensated sum per entry.
 */
int oracle_padf_k(int n_R, const int *R, const double *const *C0, long n_entries, const double *kfrac, double *out,
                  int n_threads) {
  if (n_R <= 0 || n_entries <= 0) return 1;
  double *c = (double *)malloc(sizeof(double) * n_R), *sn = (double *)malloc(sizeof(double) * n_R);
  if (!c || !sn) return 1;
  const double two_pi = 6.283185307179586476925286766559;
  for (int r = 0; r < n_R; ++r) {
    const double x = kfrac[0] * R[3 * r] + kfrac[1] * R[3 * r + 1] + kfrac[2] * R[3 * r + 2];
    c[r] = cos(two_pi * x);
    sn[r] = sin(two_pi * x);
  }
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(static) num_threads(n_threads)
  for (long e = 0; e < n_entries; ++e) {
    nsum_t sr = {0, 0}, si = {0, 0};
    for (int r = 0; r < n_R; ++r) {
      nsum_add(&sr, C0[r][e] * c[r]);
      nsum_add(&si, C0[r][e] * sn[r]);
    }
    out[2 * e] = nsum_get(&sr);
    out[2 * e + 1] = nsum_get(&si);
  }
  free(c);
  free(sn);
  return 0;
}

/* ---------------------------------------- AO -> MO fit coefficients -- */
/*
 * Fit coefficients of the orbital pair psi*_i(k) psi_a(k+q) from the
 * k-dependent pair-atomic (PADF) fit coefficients, Sec. 2.2:
 *
 * - PADF: a product of basis functions mu on atom A and nu on atom B is
 *   fitted by fit functions on A and on B only;
 * - in reciprocal space, with C_{nu mu alpha}(k) the lattice sum of the
 *   cell-pair coefficients times e^{i k.dR} (the k-dependent coefficients),
 *     chi*_mu(k) chi_nu(k+q) = sum_gamma B^{mu nu}_gamma f_gamma(q),
 *     B^{mu nu}_gamma = [gamma on atom(mu)] C_{nu mu gamma}(k+q)
 *                     + [gamma on atom(nu)] conj(C_{mu nu gamma}(k));
 * - with the KS states psi_n(k) = sum_mu c_{mu n}(k) chi_mu(k) the pair
 *   coefficients are
 *     C_{gamma, ia}(q, k) = sum_{mu, nu} conj(c_{mu i}(k)) c_{nu a}(k+q)
 *                           B^{mu nu}_gamma,
 *   i an occupied state at k, a a virtual state at k+q (the pair convention
 *   of oracle_chi0).
 *
 * Layout.  Atoms carry nb[A] basis and nf[A] fit functions, numbered atom by
 * atom.  The PADF array of a k-point is n_bas x S, S = sum_A nb[A] nf[A]:
 * row nu, column s(mu, alpha) = sum_{A' < A} nb[A'] nf[A']
 * + (mu - first basis function of A) nf[A] + alpha_loc, A = atom(mu),
 * alpha_loc the index of alpha among A's fit functions.  MO arrays are
 * n_bas x n_mo, occupied columns 0..n_occ-1, virtual columns n_occ..
 * n_occ+n_virt-1.  padf_k / mo_k belong to k, padf_kq / mo_kq to k+q.
 *
 * Output: entries (gamma, t), t = i*n_virt + a.  With entries == NULL all
 * n_aux x n_occ*n_virt values are written row-major into out; otherwise
 * out[e] receives the entry (entries[2e], entries[2e+1]).  Every entry is
 * the double sum over (mu, nu) written out, B formed term by term.
 */
int oracle_ao2mo(int is_complex, int n_atoms, const int *nb, const int *nf, int n_occ, int n_virt, int n_mo,
                 const double *padf_k, const double *padf_kq, const double *mo_k, const double *mo_kq,
                 int n_entries, const int *entries, double *out, int n_threads) {
  if (n_atoms <= 0 || n_occ <= 0 || n_virt <= 0 || n_occ + n_virt > n_mo) return 1;
  int n_bas = 0, n_aux = 0, S = 0;
  for (int A = 0; A < n_atoms; ++A) {
    if (nb[A] <= 0 || nf[A] <= 0) return 1;
    n_bas += nb[A];
    n_aux += nf[A];
    S += nb[A] * nf[A];
  }
  if (n_mo > n_bas) return 1;
  int *atom_of_bas = (int *)malloc(sizeof(int) * n_bas);
  int *bas_first = (int *)malloc(sizeof(int) * n_atoms);
  int *fit_first = (int *)malloc(sizeof(int) * n_atoms);
  int *pf_first = (int *)malloc(sizeof(int) * n_atoms);
  if (!atom_of_bas || !bas_first || !fit_first || !pf_first) return 1;
  for (int A = 0, b = 0, f = 0, p = 0; A < n_atoms; ++A) {
    bas_first[A] = b;
    fit_first[A] = f;
    pf_first[A] = p;
    for (int m = 0; m < nb[A]; ++m) atom_of_bas[b + m] = A;
    b += nb[A];
    f += nf[A];
    p += nb[A] * nf[A];
  }
  const int n_ov = n_occ * n_virt;
  const long total = entries ? (long)n_entries : (long)n_aux * n_ov;
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads)
  for (long e = 0; e < total; ++e) {
    const int gamma = entries ? entries[2 * e] : (int)(e / n_ov);
    const int t = entries ? entries[2 * e + 1] : (int)(e % n_ov);
    const int i = t / n_virt, a = n_occ + t % n_virt;
    int G = 0;
    while (G + 1 < n_atoms && gamma >= fit_first[G + 1]) ++G;
    const int g_loc = gamma - fit_first[G];
    nsum_t sr = {0, 0}, si = {0, 0};
    for (int mu = 0; mu < n_bas; ++mu) {
      for (int nu = 0; nu < n_bas; ++nu) {
        double br = 0.0, bi = 0.0;
        if (atom_of_bas[mu] == G) { /* C_{nu mu gamma}(k+q) */
          const size_t x = (size_t)nu * S + pf_first[G] + (size_t)(mu - bas_first[G]) * nf[G] + g_loc;
          br += re_(padf_kq, is_complex, x);
          bi += im_(padf_kq, is_complex, x);
        }
        if (atom_of_bas[nu] == G) { /* conj(C_{mu nu gamma}(k)) */
          const size_t x = (size_t)mu * S + pf_first[G] + (size_t)(nu - bas_first[G]) * nf[G] + g_loc;
          br += re_(padf_k, is_complex, x);
          bi -= im_(padf_k, is_complex, x);
        }
        if (br == 0.0 && bi == 0.0) continue;
        const size_t xi = (size_t)mu * n_mo + i, xa = (size_t)nu * n_mo + a;
        /* conj(c_{mu i}(k)) c_{nu a}(k+q) */
        const double cr = re_(mo_k, is_complex, xi), ci = -im_(mo_k, is_complex, xi);
        const double dr = re_(mo_kq, is_complex, xa), di = im_(mo_kq, is_complex, xa);
        const double pr = cr * dr - ci * di, pi = cr * di + ci * dr;
        nsum_add(&sr, pr * br - pi * bi);
        if (is_complex) nsum_add(&si, pr * bi + pi * br);
      }
    }
    if (is_complex) {
      out[2 * e] = nsum_get(&sr);
      out[2 * e + 1] = nsum_get(&si);
    } else {
      out[e] = nsum_get(&sr);
    }
  }
  free(atom_of_bas);
  free(bas_first);
  free(fit_first);
  free(pf_first);
  return 0;
}

/* -------------------------------------------------- Hermitian Jacobi eig -- */
/*
 * Cyclic Jacobi eigendecomposition A = U diag(lam) U^H of a Hermitian matrix
 * (real symmetric when is_complex == 0).  For each off-diagonal entry
 * a_pq = r e^{i phi}: first the phase is removed with D = diag(.., e^{-i phi}
 * at q, ..), making the (p,q) entry real and positive; then the real plane
 * rotation of Golub & Van Loan (Matrix Computations, Alg. 8.5.1/8.5.2,
 * "symmetric Schur decomposition") zeroes it.  U accumulates D and J.
 * Sweeps stop when the off-diagonal Frobenius norm is below tol times the
 * full Frobenius norm.  A is not modified; lam (n) and U (n x n) are written.
 * Returns the number of sweeps used, or -5 when max_sweeps is exceeded.
 */
int oracle_jacobi_eigh(int is_complex, int n, const double *A_in, double *lam, double *U_out, int max_sweeps,
                       double tol) {
  if (n <= 0) return -1;
  const int c = is_complex ? 2 : 1;
  double *A = (double *)malloc(sizeof(double) * (size_t)n * n * 2);
  double *U = (double *)malloc(sizeof(double) * (size_t)n * n * 2);
  if (!A || !U) return -1;
  /* work in complex form throughout for one code path */
  for (size_t i = 0; i < (size_t)n * n; ++i) {
    A[2 * i] = A_in[c * i];
    A[2 * i + 1] = is_complex ? A_in[2 * i + 1] : 0.0;
    U[2 * i] = 0.0;
    U[2 * i + 1] = 0.0;
  }
  for (int i = 0; i < n; ++i) {
    U[2 * ((size_t)i * n + i)] = 1.0;
    A[2 * ((size_t)i * n + i) + 1] = 0.0; /* Hermitian: real diagonal */
  }
  nsum_t fro = {0, 0};
  for (size_t i = 0; i < (size_t)n * n; ++i) nsum_add(&fro, A[2 * i] * A[2 * i] + A[2 * i + 1] * A[2 * i + 1]);
  double norm = sqrt(nsum_get(&fro));
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    nsum_t off = {0, 0};
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        size_t k = (size_t)p * n + q;
        nsum_add(&off, 2.0 * (A[2 * k] * A[2 * k] + A[2 * k + 1] * A[2 * k + 1]));
      }
    if (sqrt(nsum_get(&off)) <= tol * norm) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        size_t kpq = (size_t)p * n + q;
        double xr = A[2 * kpq], xi = A[2 * kpq + 1];
        double r = hypot(xr, xi);
        if (r == 0.0) continue;
        /* phase e^{-i phi} applied to column q, e^{+i phi} to row q */
        double er = xr / r, ei = -xi / r; /* e^{-i phi} */
        for (int i = 0; i < n; ++i) {     /* column q: A[i][q] *= e^{-i phi} */
          size_t k = (size_t)i * n + q;
          double ar = A[2 * k], ai = A[2 * k + 1];
          A[2 * k] = ar * er - ai * ei;
          A[2 * k + 1] = ar * ei + ai * er;
          double ur = U[2 * k], ui = U[2 * k + 1];
          U[2 * k] = ur * er - ui * ei;
          U[2 * k + 1] = ur * ei + ui * er;
        }
        for (int i = 0; i < n; ++i) { /* row q: A[q][i] *= e^{+i phi} */
          size_t k = (size_t)q * n + i;
          double ar = A[2 * k], ai = A[2 * k + 1];
          A[2 * k] = ar * er + ai * ei;
          A[2 * k + 1] = -ar * ei + ai * er;
        }
        /* now A[p][q] = A[q][p] = r, real */
        double app = A[2 * ((size_t)p * n + p)], aqq = A[2 * ((size_t)q * n + q)];
        double apq = A[2 * kpq];
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        /* A <- J^T A J with J_pp = J_qq = cs, J_pq = sn, J_qp = -sn */
        for (int i = 0; i < n; ++i) { /* columns p, q */
          size_t kp = (size_t)i * n + p, kq = (size_t)i * n + q;
          double pr = A[2 * kp], pi = A[2 * kp + 1], qr = A[2 * kq], qi = A[2 * kq + 1];
          A[2 * kp] = cs * pr - sn * qr;
          A[2 * kp + 1] = cs * pi - sn * qi;
          A[2 * kq] = sn * pr + cs * qr;
          A[2 * kq + 1] = sn * pi + cs * qi;
          double upr = U[2 * kp], upi = U[2 * kp + 1], uqr = U[2 * kq], uqi = U[2 * kq + 1];
          U[2 * kp] = cs * upr - sn * uqr;
          U[2 * kp + 1] = cs * upi - sn * uqi;
          U[2 * kq] = sn * upr + cs * uqr;
          U[2 * kq + 1] = sn * upi + cs * uqi;
        }
        for (int i = 0; i < n; ++i) { /* rows p, q */
          size_t kp = (size_t)p * n + i, kq = (size_t)q * n + i;
          double pr = A[2 * kp], pi = A[2 * kp + 1], qr = A[2 * kq], qi = A[2 * kq + 1];
          A[2 * kp] = cs * pr - sn * qr;
          A[2 * kp + 1] = cs * pi - sn * qi;
          A[2 * kq] = sn * pr + cs * qr;
          A[2 * kq + 1] = sn * pi + cs * qi;
        }
        A[2 * kpq] = A[2 * kpq + 1] = 0.0;
        A[2 * ((size_t)q * n + p)] = A[2 * ((size_t)q * n + p) + 1] = 0.0;
        A[2 * ((size_t)p * n + p) + 1] = 0.0;
        A[2 * ((size_t)q * n + q) + 1] = 0.0;
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[2 * ((size_t)i * n + i)];
  for (size_t i = 0; i < (size_t)n * n; ++i) {
    U_out[c * i] = U[2 * i];
    if (is_complex) U_out[2 * i + 1] = U[2 * i + 1];
  }
  free(A);
  free(U);
  return sweep < max_sweeps ? sweep : -5;
}

/* --------------------------------------------------------- V^(1/2) ----- */
/*
 * Square root of the Hermitian positive-definite fit-basis Coulomb matrix
 * (Sec. 2.1, v^(1/2)(q); Algorithm 1, "eval. V^0.5(q)"):
 *   V = U diag(lam) U^H  ->  V^(1/2) = U diag(sqrt(lam)) U^H.
 * Returns 4 if an eigenvalue is not positive, 5 if Jacobi did not converge.
 */
int oracle_vhalf(int is_complex, int n, const double *V, double *Vh) {
  const int c = is_complex ? 2 : 1;
  double *lam = (double *)malloc(sizeof(double) * n);
  double *U = (double *)malloc(sizeof(double) * (size_t)n * n * c);
  int rc = oracle_jacobi_eigh(is_complex, n, V, lam, U, 100, 1e-14);
  if (rc < 0) {
    free(lam);
    free(U);
    return 5;
  }
  for (int i = 0; i < n; ++i)
    if (!(lam[i] > 0.0)) {
      free(lam);
      free(U);
      return 4;
    }
  for (int P = 0; P < n; ++P)
    for (int Q = 0; Q < n; ++Q) {
      nsum_t sr = {0, 0}, si = {0, 0};
      for (int m = 0; m < n; ++m) {
        double s = sqrt(lam[m]);
        size_t ip = (size_t)P * n + m, iq = (size_t)Q * n + m;
        double ur = re_(U, is_complex, ip), ui = im_(U, is_complex, ip);
        double vr = re_(U, is_complex, iq), vi = -im_(U, is_complex, iq); /* conj(U[Q][m]) */
        nsum_add(&sr, s * (ur * vr - ui * vi));
        if (is_complex) nsum_add(&si, s * (ur * vi + ui * vr));
      }
      size_t o = (size_t)P * n + Q;
      if (is_complex) {
        Vh[2 * o] = nsum_get(&sr);
        Vh[2 * o + 1] = nsum_get(&si);
      } else {
        Vh[o] = nsum_get(&sr);
      }
    }
  free(lam);
  free(U);
  return 0;
}

/* -------------------------------------------------------- matmul ------- */
/* C = A B, n x n, plain triple loop with compensated sums. */
static void matmul(int is_c, int n, const double *A, const double *B, double *Cm, int n_threads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      nsum_t sr = {0, 0}, si = {0, 0};
      for (int k = 0; k < n; ++k) {
        size_t ia = (size_t)i * n + k, ib = (size_t)k * n + j;
        double ar = re_(A, is_c, ia), ai = im_(A, is_c, ia), br = re_(B, is_c, ib), bi = im_(B, is_c, ib);
        nsum_add(&sr, ar * br);
        if (is_c) {
          nsum_add(&sr, -ai * bi);
          nsum_add(&si, ar * bi);
          nsum_add(&si, ai * br);
        }
      }
      size_t o = (size_t)i * n + j;
      if (is_c) {
        Cm[2 * o] = nsum_get(&sr);
        Cm[2 * o + 1] = nsum_get(&si);
      } else {
        Cm[o] = nsum_get(&sr);
      }
    }
}

/*
 * Symmetrised response Z = Pi = V^(1/2) chi V^(1/2) (Sec. 2.1, working
 * equation; Algorithm 1, "Z = V^0.5 P V^0.5").  All n x n.
 */
int oracle_sandwich(int is_complex, int n, const double *Vh, const double *chi, double *Pi, int n_threads) {
  const int c = is_complex ? 2 : 1;
  double *T = (double *)malloc(sizeof(double) * (size_t)n * n * c);
  if (!T) return 1;
  if (n_threads < 1) n_threads = 1;
  matmul(is_complex, n, chi, Vh, T, n_threads);
  matmul(is_complex, n, Vh, T, Pi, n_threads);
  free(T);
  return 0;
}

/* --------------------------------------------------------- log det ----- */
/*
 * ln det(1 - Pi) and Tr Pi (Sec. 2.1 working equation; Algorithm 1, the RPA
 * integrand) from an unblocked Cholesky factorisation 1 - Pi = L L^H of the
 * Hermitian positive-definite matrix M = 1 - Pi.
 *
 * Column j of the factor: u_j = M_jj - 1 - sum_{k<j} |L_jk|^2 is the pivot
 * minus one (formed without adding the 1, so that pivots close to 1 keep
 * their digits), L_jj = sqrt(1 + u_j), L_ij = (M_ij - sum_{k<j} L_ik
 * conj(L_jk)) / L_jj for i > j, and ln det M = sum_j ln L_jj^2 =
 * sum_j log1p(u_j).  Only the lower triangle of Pi is read.
 * Returns 4 if a pivot is not positive.
 */
int oracle_logdet_cholesky(int is_complex, int n, const double *Pi, double *lndet, double *trPi) {
  double *L = (double *)calloc((size_t)n * n * 2, sizeof(double));
  if (!L) return 1;
  nsum_t ld = {0, 0}, tr = {0, 0};
  for (int j = 0; j < n; ++j) nsum_add(&tr, re_(Pi, is_complex, (size_t)j * n + j));
  for (int j = 0; j < n; ++j) {
    nsum_t u = {0, 0};
    nsum_add(&u, -re_(Pi, is_complex, (size_t)j * n + j));
    for (int k = 0; k < j; ++k) {
      size_t jk = (size_t)j * n + k;
      nsum_add(&u, -(L[2 * jk] * L[2 * jk] + L[2 * jk + 1] * L[2 * jk + 1]));
    }
    double uj = nsum_get(&u);
    if (!(1.0 + uj > 0.0)) {
      free(L);
      return 4;
    }
    double ljj = sqrt(1.0 + uj);
    nsum_add(&ld, log1p(uj));
    L[2 * ((size_t)j * n + j)] = ljj;
    for (int i = j + 1; i < n; ++i) {
      size_t ij = (size_t)i * n + j;
      nsum_t sr = {0, 0}, si = {0, 0};
      nsum_add(&sr, -re_(Pi, is_complex, ij));
      nsum_add(&si, -im_(Pi, is_complex, ij));
      for (int k = 0; k < j; ++k) {
        size_t ik = (size_t)i * n + k, jk = (size_t)j * n + k;
        double ar = L[2 * ik], ai = L[2 * ik + 1], br = L[2 * jk], bi = -L[2 * jk + 1];
        nsum_add(&sr, -(ar * br - ai * bi));
        nsum_add(&si, -(ar * bi + ai * br));
      }
      L[2 * ij] = nsum_get(&sr) / ljj;
      L[2 * ij + 1] = nsum_get(&si) / ljj;
    }
  }
  *lndet = nsum_get(&ld);
  *trPi = nsum_get(&tr);
  free(L);
  return 0;
}

/*
 * Cross-check: ln |det M| of a general n x n matrix M by LU factorisation with
 * partial pivoting (Doolittle, Golub & Van Loan Alg. 3.4.1).  M is copied.
 */
int oracle_logabsdet_lu(int is_complex, int n, const double *M_in, double *ln_abs_det) {
  double *M = (double *)malloc(sizeof(double) * (size_t)n * n * 2);
  if (!M) return 1;
  for (size_t i = 0; i < (size_t)n * n; ++i) {
    M[2 * i] = re_(M_in, is_complex, i);
    M[2 * i + 1] = im_(M_in, is_complex, i);
  }
  nsum_t acc = {0, 0};
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = -1.0;
    for (int i = k; i < n; ++i) {
      size_t ik = (size_t)i * n + k;
      double a = hypot(M[2 * ik], M[2 * ik + 1]);
      if (a > best) {
        best = a;
        piv = i;
      }
    }
    if (best == 0.0) {
      free(M);
      *ln_abs_det = -INFINITY;
      return 0;
    }
    if (piv != k)
      for (int j = 0; j < n; ++j) {
        size_t a = (size_t)k * n + j, b = (size_t)piv * n + j;
        double tr = M[2 * a], ti = M[2 * a + 1];
        M[2 * a] = M[2 * b];
        M[2 * a + 1] = M[2 * b + 1];
        M[2 * b] = tr;
        M[2 * b + 1] = ti;
      }
    size_t kk = (size_t)k * n + k;
    double pr = M[2 * kk], pi = M[2 * kk + 1];
    nsum_add(&acc, log(hypot(pr, pi)));
    double den = pr * pr + pi * pi;
    for (int i = k + 1; i < n; ++i) {
      size_t ik = (size_t)i * n + k;
      double ar = M[2 * ik], ai = M[2 * ik + 1];
      double lr = (ar * pr + ai * pi) / den, li = (ai * pr - ar * pi) / den; /* a / p */
      M[2 * ik] = lr;
      M[2 * ik + 1] = li;
      for (int j = k + 1; j < n; ++j) {
        size_t ij = (size_t)i * n + j, kj = (size_t)k * n + j;
        double br = M[2 * kj], bi = M[2 * kj + 1];
        M[2 * ij] -= lr * br - li * bi;
        M[2 * ij + 1] -= lr * bi + li * br;
      }
    }
  }
  *ln_abs_det = nsum_get(&acc);
  free(M);
  return 0;
}

/* ------------------------------------------------------ quadrature ----- */
/*
 * RPA correlation energy from the integrand table (Sec. 2.6, the (q, omega)
 * double sum; Sec. 2.1 working equation with the sign reading
 * E = +(1/2 pi) int d omega sum_q w_q [ln det(1 - Pi) + Tr Pi]):
 *
 *   E_c = (1/2 pi) sum_w zeta_w sum_q w_q eps[q][w],
 *
 * eps[q][w] = ln det(1 - Pi(q, i omega_w)) + Tr Pi(q, i omega_w), stored
 * [n_q][n_w].  The q-sum is formed per frequency first (e_omega), then the
 * frequency sum, both compensated.
 */
int oracle_energy_sum(int n_q, int n_w, const double *w_q, const double *zeta_w, const double *eps, double *Ec) {
  nsum_t E = {0, 0};
  for (int w = 0; w < n_w; ++w) {
    nsum_t e = {0, 0};
    for (int q = 0; q < n_q; ++q) nsum_add(&e, w_q[q] * eps[(size_t)q * n_w + w]);
    nsum_add(&E, zeta_w[w] * nsum_get(&e));
  }
  *Ec = nsum_get(&E) / (2.0 * M_PI);
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
