// Frequency-batched chi0: the plan (host code).
//
// chi0_PQ(q, w) = sum_t conj(C_Pt) C_Qt d_t(w), d_t(w) = -4 D_t / (D_t^2 + w^2)
// (Sec. 2.2), evaluated at every node w of the frequency grid.  Algorithm 1
// of the paper rebuilds the whole contraction for each frequency.  Because
// d_t(w) depends on t only through the transition energy D_t, and is a
// smooth function of D with its poles at D = +-i w, its restriction to a
// narrow window of D is numerically of low rank across the n_w nodes: on a
// window whose ends differ by a factor ~1.5 about nine terms reach 1e-10 of
// the window's largest weight, for any set of nodes.  So the transitions of a
// q are split into windows ("bins") of D, and within bin b
//   d(D, w) ~= sum_r coef_b[r][w] d(D, w_{s(b,r)})   (D in bin b),
// an interpolative decomposition over a subset of the nodes themselves (the
// skeleton frequencies s(b, r)).  Then
//   chi0(w) ~= sum_b sum_r coef_b[r][w] X_{b,r},
//   X_{b,r} = sum_{t in bin b} conj(C_Pt) C_Qt d_t(w_{s(b,r)}),
// i.e. R_b contractions over the bin's transitions instead of n_w: the
// imaginary-time idea the paper's conclusions point to (a few basis functions
// of D shared by all frequencies) in a form that is exact at the skeleton
// nodes and whose error is controlled per bin.
//
// The skeleton and its coefficients come from a Householder QR with column
// pivoting (Businger and Golub, 1965) of the matrix of column-scaled weights
// d(D_i, w)/max_i |d(D_i, w)| on Chebyshev points D_i of the bin; the rank is
// the smallest whose residual, checked on a dense grid of the bin, is below
// FREQ_TOL of every column's maximum and whose coefficient sum stays below
// FREQ_AMP (it multiplies the split-precision error of the X_{b,r}).  Since
// all d_t(w) of a frequency have one sign, a relative error e of every weight
// bounds the error of chi0(w) by e |chi0(w)| in the Loewner order.  Bins are
// geometric in D between the job's smallest and largest transition energy;
// the bin ratio is chosen among a few candidates by the modelled work
// sum_b R_b K_b (K_b: transitions of bin b), and the plan is used only when it
// saves work over n_w full contractions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <thread>
#include <vector>

#include "rpa_internal.h"
#include "rpa_runtime.h"

namespace rpa {
namespace {

constexpr int N_FIT = 64;     // Chebyshev points per bin for the decomposition
constexpr int N_CHECK = 601;  // points per bin on which the residual is checked

double weight(double D, double w) { return -4.0 * D / (D * D + w * w); }

// Householder QR with column pivoting of the m x n matrix A (row-major,
// m >= n), in place: on return the upper triangle holds R, piv the column
// order (A P = Q R).
void qrcp(int m, int n, std::vector<double>& A, std::vector<int>& piv) {
  piv.resize(n);
  for (int j = 0; j < n; ++j) piv[j] = j;
  std::vector<double> norm2(n, 0.0), v(m);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) norm2[j] += A[(size_t)i * n + j] * A[(size_t)i * n + j];
  for (int k = 0; k < n && k < m; ++k) {
    // column of largest remaining norm
    int p = k;
    for (int j = k + 1; j < n; ++j)
      if (norm2[j] > norm2[p]) p = j;
    if (p != k) {
      for (int i = 0; i < m; ++i) std::swap(A[(size_t)i * n + k], A[(size_t)i * n + p]);
      std::swap(norm2[k], norm2[p]);
      std::swap(piv[k], piv[p]);
    }
    // Householder reflector of A[k:, k]
    double s = 0.0;
    for (int i = k; i < m; ++i) s += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    const double alpha = A[(size_t)k * n + k] >= 0.0 ? -sqrt(s) : sqrt(s);
    if (s == 0.0) continue;
    for (int i = k; i < m; ++i) v[i] = A[(size_t)i * n + k];
    v[k] -= alpha;
    double vn = 0.0;
    for (int i = k; i < m; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    for (int j = k; j < n; ++j) {
      double d = 0.0;
      for (int i = k; i < m; ++i) d += v[i] * A[(size_t)i * n + j];
      d *= 2.0 / vn;
      for (int i = k; i < m; ++i) A[(size_t)i * n + j] -= d * v[i];
    }
    // downdate the remaining column norms (recomputed: the matrices are small)
    for (int j = k + 1; j < n; ++j) {
      double t = 0.0;
      for (int i = k + 1; i < m; ++i) t += A[(size_t)i * n + j] * A[(size_t)i * n + j];
      norm2[j] = t;
    }
  }
}

struct BinFit {
  int rank = 0;
  std::vector<int> skel;     // [rank] node indices
  std::vector<double> coef;  // [rank][n_w], unscaled: d(., w) ~= sum_r coef[r][w] d(., w_skel[r])
  double err = 0.0;          // residual / column maximum on the check grid
  double amp = 0.0;          // max_w sum_r |scaled coefficient|
};

// Interpolative decomposition of the weights on [lo, hi] across the nodes.
BinFit fit_bin(double lo, double hi, const double* omega, int n_w, double tol, double amp_max,
               int n_check = N_CHECK) {
  BinFit f;
  std::vector<double> x(N_FIT), xc(n_check), s(n_w, 0.0);
  for (int i = 0; i < N_FIT; ++i)
    x[i] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * cos(M_PI * (i + 0.5) / N_FIT);
  for (int i = 0; i < n_check; ++i) xc[i] = lo + (hi - lo) * (double)i / (n_check - 1);
  // column scale: the largest |d| of each node over the bin (check grid and fit points)
  std::vector<double> Mc((size_t)n_check * n_w);
  for (int i = 0; i < n_check; ++i)
    for (int w = 0; w < n_w; ++w) {
      Mc[(size_t)i * n_w + w] = weight(xc[i], omega[w]);
      s[w] = std::max(s[w], fabs(Mc[(size_t)i * n_w + w]));
    }
  for (int w = 0; w < n_w; ++w)
    for (int i = 0; i < N_FIT; ++i) s[w] = std::max(s[w], fabs(weight(x[i], omega[w])));
  for (int i = 0; i < n_check; ++i)
    for (int w = 0; w < n_w; ++w) Mc[(size_t)i * n_w + w] /= s[w];
  std::vector<double> A((size_t)N_FIT * n_w);
  for (int i = 0; i < N_FIT; ++i)
    for (int w = 0; w < n_w; ++w) A[(size_t)i * n_w + w] = weight(x[i], omega[w]) / s[w];
  std::vector<int> piv;
  std::vector<double> R = A;
  qrcp(N_FIT, n_w, R, piv);
  const int kmax = std::min(n_w, N_FIT);
  // scaled coefficients T ([r][w], original column order) of the rank-r
  // decomposition, T = R11^-1 R12 for the non-skeleton columns; false if R11
  // is singular
  auto coeffs = [&](int r, std::vector<double>& T) -> bool {
    T.assign((size_t)r * n_w, 0.0);
    for (int k = 0; k < r; ++k) T[(size_t)k * n_w + piv[k]] = 1.0;
    std::vector<double> y(r);
    for (int c = r; c < n_w; ++c) {
      for (int k = r - 1; k >= 0; --k) {
        double acc = R[(size_t)k * n_w + c];
        for (int l = k + 1; l < r; ++l) acc -= R[(size_t)k * n_w + l] * y[l];
        const double dkk = R[(size_t)k * n_w + k];
        if (dkk == 0.0) return false;
        y[k] = acc / dkk;
      }
      for (int k = 0; k < r; ++k) T[(size_t)k * n_w + piv[c]] = y[k];
    }
    return true;
  };
  // residual on the check grid and the coefficient sum; false when the rank fails the bars
  auto passes = [&](int r, std::vector<double>& T, double& err, double& amp) -> bool {
    if (!coeffs(r, T)) return false;
    amp = 0.0;
    for (int w = 0; w < n_w; ++w) {
      double a = 0.0;
      for (int k = 0; k < r; ++k) a += fabs(T[(size_t)k * n_w + w]);
      amp = std::max(amp, a);
    }
    if (amp > amp_max) return false;
    err = 0.0;
    for (int i = 0; i < n_check; ++i) {
      const double* m = &Mc[(size_t)i * n_w];
      for (int w = 0; w < n_w; ++w) {
        double v = m[w];
        for (int k = 0; k < r; ++k) v -= T[(size_t)k * n_w + w] * m[piv[k]];
        err = std::max(err, fabs(v));
        if (err > tol) return false;
      }
    }
    return true;
  };
  // first guess from the pivots' decay, then the smallest rank that passes
  const double r00 = fabs(R[0]);
  int r0 = kmax;
  for (int k = 1; k < kmax; ++k)
    if (fabs(R[(size_t)k * n_w + k]) <= tol * r00) {
      r0 = k;
      break;
    }
  std::vector<double> T, Tbest;
  double err = 0.0, amp = 0.0, ebest = 0.0, abest = 0.0;
  int rbest = 0;
  for (int r = r0; r <= kmax; ++r)
    if (passes(r, T, err, amp)) {
      rbest = r;
      Tbest = T;
      ebest = err;
      abest = amp;
      break;
    }
  while (rbest > 1 && passes(rbest - 1, T, err, amp)) {
    --rbest;
    Tbest = T;
    ebest = err;
    abest = amp;
  }
  if (rbest > 0) {
    f.rank = rbest;
    f.err = ebest;
    f.amp = abest;
    f.skel.assign(piv.begin(), piv.begin() + rbest);
    f.coef.assign((size_t)rbest * n_w, 0.0);
    for (int k = 0; k < rbest; ++k)
      for (int w = 0; w < n_w; ++w) f.coef[(size_t)k * n_w + w] = Tbest[(size_t)k * n_w + w] * s[w] / s[piv[k]];
    return f;
  }
  // no truncation reaches the bar: every node is its own skeleton
  f.rank = n_w;
  f.err = 0.0;
  f.amp = 1.0;
  f.skel.resize(n_w);
  f.coef.assign((size_t)n_w * n_w, 0.0);
  for (int w = 0; w < n_w; ++w) {
    f.skel[w] = w;
    f.coef[(size_t)w * n_w + w] = 1.0;
  }
  return f;
}

// Transition-energy window [lo, hi] of the job (every pair of every q).
bool delta_range(const rpa_job* j, const double* eo, const double* ev, double& lo, double& hi) {
  lo = std::numeric_limits<double>::infinity();
  hi = -lo;
  std::vector<double> omin(j->n_kpts), omax(j->n_kpts), vmin(j->n_kpts), vmax(j->n_kpts);
  for (int k = 0; k < j->n_kpts; ++k) {
    omin[k] = *std::min_element(eo + (size_t)k * j->n_occ, eo + (size_t)(k + 1) * j->n_occ);
    omax[k] = *std::max_element(eo + (size_t)k * j->n_occ, eo + (size_t)(k + 1) * j->n_occ);
    vmin[k] = *std::min_element(ev + (size_t)k * j->n_virt, ev + (size_t)(k + 1) * j->n_virt);
    vmax[k] = *std::max_element(ev + (size_t)k * j->n_virt, ev + (size_t)(k + 1) * j->n_virt);
  }
  for (long p = 0; p < (long)j->n_q * j->n_k; ++p) {
    lo = std::min(lo, vmin[j->pair_kq[p]] - omax[j->pair_k[p]]);
    hi = std::max(hi, vmax[j->pair_kq[p]] - omin[j->pair_k[p]]);
  }
  return isfinite(lo) && isfinite(hi) && lo > 0.0;
}

// Virtual energies of every k-point in ascending order (for the counts).
std::vector<double> sorted_virt(const rpa_job* j, const double* ev) {
  std::vector<double> s(ev, ev + (size_t)j->n_kpts * j->n_virt);
  for (int k = 0; k < j->n_kpts; ++k)
    std::sort(s.begin() + (size_t)k * j->n_virt, s.begin() + (size_t)(k + 1) * j->n_virt);
  return s;
}

// Number of a with ev_sorted[a] - e_i >= edge (the device's bin test, same
// FP64 subtraction; monotone in a).
int count_ge(const double* evs, int n, double e_i, double edge) {
  int lo = 0, hi = n;  // first index with evs[idx] - e_i >= edge
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (evs[mid] - e_i >= edge)
      hi = mid;
    else
      lo = mid + 1;
  }
  return n - lo;
}

}  // namespace

void freq_parallel_q(int n_q, const std::function<void(int)>& fn) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::min<int>(n_q, (int)std::min(8u, hw));
  if (nt <= 1) {
    for (int q = 0; q < n_q; ++q) fn(q);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int q = t; q < n_q; q += nt) fn(q);
    });
  for (auto& x : th) x.join();
}

int freq_bin_of(const FreqPlan& p, double D) {
  int b = 0;
  while (b < p.n_bins - 1 && D >= p.edges[b]) ++b;
  return b;
}

void freq_counts(const rpa_job* j, const FreqPlan& p, int q, const double* eo, const double* evs, int* cnt) {
  const int nb = p.n_bins;
  for (int jj = 0; jj < j->n_k; ++jj) {
    const long pr = (long)q * j->n_k + jj;
    const double* e_o = eo + (size_t)j->pair_k[pr] * j->n_occ;
    const double* e_v = evs + (size_t)j->pair_kq[pr] * j->n_virt;
    for (int i = 0; i < j->n_occ; ++i) {
      int* c = cnt + ((size_t)jj * j->n_occ + i) * nb;
      int above = j->n_virt;  // a with D >= edge[b - 1] (all for b = 0)
      for (int b = 0; b < nb; ++b) {
        const int ge_next = b + 1 < nb ? count_ge(e_v, j->n_virt, e_o[i], p.edges[b]) : 0;
        c[b] = above - ge_next;
        above = ge_next;
      }
    }
  }
}

bool freq_plan_build(const rpa_job* j, const double* eo, const double* ev, int mode, FreqPlan* out,
                     std::vector<int>* counts) {
  FreqPlan& P = *out;
  P = FreqPlan{};
  if (mode == 1 || j->n_w < 2 || j->n_w > 32) return false;
  if ((long long)j->n_k * j->n_occ * j->n_virt + 16LL * FREQ_MAX_BINS >= (1LL << 30)) return false;
  double lo, hi;
  if (!delta_range(j, eo, ev, lo, hi)) return false;
  const std::vector<double> evs = sorted_virt(j, ev);
  const double total = (double)j->n_q * j->n_k * j->n_occ * j->n_virt;
  auto bins_for = [&](double rho) {
    return std::min(FREQ_MAX_BINS, std::max(1, (int)ceil(log(hi / lo) / log(rho) - 1e-9)));
  };
  auto bin_ends = [&](int nb, int b, double& blo, double& bhi) {
    const double step = pow(hi / lo, 1.0 / nb);
    blo = b == 0 ? lo : lo * pow(step, b);
    bhi = b == nb - 1 ? hi : lo * pow(step, b + 1);
  };
  // The whole plan for bin ratio rho: every bin fitted, the bins' populations
  // counted over the job, the modelled work.
  auto plan_full = [&](double rho) {
    FreqPlan c;
    const int nb = bins_for(rho);
    c.n_bins = nb;
    for (int b = 0; b + 1 < nb; ++b) {
      double blo, bhi;
      bin_ends(nb, b, blo, bhi);
      c.edges[b] = bhi;
    }
    // bin populations over the whole job (the per-q counts are kept for the
    // device tables)
    std::vector<double> kb(nb, 0.0);
    const size_t per_q = (size_t)j->n_k * j->n_occ * nb;
    std::vector<int> cnt(per_q * j->n_q);
    freq_parallel_q(j->n_q, [&](int q) { freq_counts(j, c, q, eo, evs.data(), cnt.data() + per_q * q); });
    for (size_t u = 0; u < cnt.size(); ++u) kb[u % nb] += cnt[u];
    if (counts) *counts = std::move(cnt);
    double work = 0.0;
    c.rmax = 0;
    std::vector<BinFit> fits(nb);
    for (int b = 0; b < nb; ++b) {
      double blo, bhi;
      bin_ends(nb, b, blo, bhi);
      if (b > 0) blo = c.edges[b - 1];
      if (b + 1 < nb) bhi = c.edges[b];
      fits[b] = fit_bin(blo, bhi, j->omega, j->n_w, FREQ_TOL, FREQ_AMP);
      c.rank[b] = fits[b].rank;
      c.err[b] = fits[b].err;
      c.amp[b] = fits[b].amp;
      c.rmax = std::max(c.rmax, fits[b].rank);
      // each bin is padded to whole K-blocks per q (at most 15 extra values)
      work += (double)fits[b].rank * (kb[b] + (kb[b] > 0 ? 8.0 * j->n_q : 0.0));
    }
    c.work_ratio = work / (total * j->n_w);
    c.skel.assign((size_t)nb * c.rmax, -1);
    c.coef.assign((size_t)nb * c.rmax * j->n_w, 0.0);
    for (int b = 0; b < nb; ++b)
      for (int r = 0; r < fits[b].rank; ++r) {
        c.skel[(size_t)b * c.rmax + r] = fits[b].skel[r];
        for (int w = 0; w < j->n_w; ++w)
          c.coef[((size_t)b * c.rmax + r) * j->n_w + w] = fits[b].coef[(size_t)r * j->n_w + w];
      }
    return c;
  };
  // Candidate ratios are screened by the mean rank of five sample bins
  // (fitted against a coarse check grid) and the padding of their bin count,
  // assuming equal populations; only the most promising is planned in full
  // (the fits and the population counts of every candidate in full took
  // ~60 ms on the slab job).
  const double ratios[] = {1.08, 1.1, 1.12, 1.15, 1.2, 1.25, 1.3, 1.5, 1.75, 2.1, 3.0};
  std::vector<std::pair<double, double>> est;  // (modelled work, rho)
  for (double rho : ratios) {
    const int nb = bins_for(rho);
    double r = 0.0;
    int ns = 0;
    for (int b : {0, nb / 4, nb / 2, (3 * nb) / 4, nb - 1}) {
      double blo, bhi;
      bin_ends(nb, b, blo, bhi);
      r += fit_bin(blo, bhi, j->omega, j->n_w, FREQ_TOL, FREQ_AMP, 101).rank;
      ++ns;
    }
    est.push_back({r / ns * (1.0 + 8.0 * j->n_q * nb / total), rho});
  }
  std::stable_sort(est.begin(), est.end(),
                   [](const std::pair<double, double>& a, const std::pair<double, double>& b) { return a.first < b.first; });
  P = plan_full(est[0].second);
  P.dlo = lo;
  P.dhi = hi;
  if ((size_t)P.n_bins * P.rmax * j->n_w * sizeof(double) > 48 * 1024) {  // coefficients of the reduction
    P.n_bins = 0;
    return false;
  }
  if (mode != 2 && P.work_ratio > 0.9) {  // no gain: contract every frequency
    P.n_bins = 0;
    return false;
  }
  return P.n_bins > 0;
}


void freq_bin_q(const rpa_job* j, const FreqPlan& p, int q, const double* eo, const double* evs, BinQHost& h,
                std::vector<int>& img, const int* counts) {
  const int nb = p.n_bins, tpk = j->is_complex ? 8 : 16;
  const long nrow = (long)j->n_k * j->n_occ;
  std::vector<int> own;
  if (!counts) {
    own.resize((size_t)nrow * nb);
    freq_counts(j, p, q, eo, evs, own.data());
    counts = own.data();
  }
  const int* cnt = counts;
  long K[FREQ_MAX_BINS] = {};
  for (long r = 0; r < nrow; ++r)
    for (int b = 0; b < nb; ++b) K[b] += cnt[(size_t)r * nb + b];
  h.tb0[0] = 0;
  for (int b = 0; b < nb; ++b) h.tb0[b + 1] = h.tb0[b] + (int)((K[b] + tpk - 1) / tpk * tpk);
  for (int b = nb + 1; b <= FREQ_MAX_BINS; ++b) h.tb0[b] = h.tb0[nb];
  h.Kt = h.tb0[nb];
  h.Kr = j->is_complex ? 2 * h.Kt : h.Kt;
  std::vector<int> parts;
  for (int b = 0; b < nb; ++b)
    for (int u = h.tb0[b]; u < h.tb0[b + 1]; u += FREQ_PART) {
      parts.push_back(b);
      parts.push_back(u);
      parts.push_back(std::min(u + FREQ_PART, h.tb0[b + 1]));
    }
  h.n_parts = (int)parts.size() / 3;
  img.assign((size_t)2 * nrow * nb + parts.size() + FREQ_MAX_BINS, 0);
  long run[FREQ_MAX_BINS];
  for (int b = 0; b < nb; ++b) run[b] = h.tb0[b];
  for (long r = 0; r < nrow; ++r)
    for (int b = 0; b < nb; ++b) {
      img[(size_t)r * nb + b] = (int)run[b];
      img[(size_t)(nrow + r) * nb + b] = cnt[(size_t)r * nb + b];
      run[b] += cnt[(size_t)r * nb + b];
    }
  std::copy(parts.begin(), parts.end(), img.begin() + (size_t)2 * nrow * nb);
  for (int b = 0; b < nb; ++b) img[(size_t)2 * nrow * nb + parts.size() + b] = p.rank[b];
}

void freq_meta_d(const rpa_job* j, const FreqPlan& p, std::vector<double>& img) {
  const size_t nbr = (size_t)p.n_bins * p.rmax;
  img.assign(nbr + nbr * j->n_w, 0.0);
  for (size_t i = 0; i < nbr; ++i) img[i] = p.skel[i] >= 0 ? j->omega[p.skel[i]] : 0.0;
  std::copy(p.coef.begin(), p.coef.end(), img.begin() + nbr);
}

}  // namespace rpa

// ============================================================== C ABI =====

extern "C" rpa_status rpa_freq_plan(const rpa_job* job, int mode, int* n_bins, double* edges, int* rank,
                                    int* skel, double* coef, double* err, double* work_ratio) {
  char msg[256];
  if (!job || rpa::validate_job(job, msg, sizeof msg)) return RPA_E_INVAL;
  if (job->mem != RPA_MEM_HOST || mode < 0 || mode > 2) return RPA_E_INVAL;
  rpa::FreqPlan p;
  rpa::freq_plan_build(job, job->eps_occ, job->eps_virt, mode, &p);
  if (n_bins) *n_bins = p.n_bins;
  if (work_ratio) *work_ratio = p.n_bins ? p.work_ratio : 1.0;
  for (int b = 0; b < p.n_bins; ++b) {
    if (edges && b + 1 < p.n_bins) edges[b] = p.edges[b];
    if (rank) rank[b] = p.rank[b];
    if (err) err[b] = p.err[b];
    for (int r = 0; r < job->n_w; ++r) {
      const bool in = r < p.rank[b];
      if (skel) skel[(size_t)b * job->n_w + r] = in ? p.skel[(size_t)b * p.rmax + r] : -1;
      for (int w = 0; w < job->n_w && coef; ++w)
        coef[((size_t)b * job->n_w + r) * job->n_w + w] = in ? p.coef[((size_t)b * p.rmax + r) * job->n_w + w] : 0.0;
    }
  }
  return RPA_OK;
}
