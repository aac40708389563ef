// Periodic projector (Sec. 2.3) on GB300: S(k) = U D U^H, R(k) = Theta(D(k) -
// eps_d), R~ = prod_k R(k), T(k) = U(k) R~ U(k)^H, c~(k) = T(k) c(k).
//
// Eigendecomposition: one-sided (Hestenes) Jacobi on the columns of W = S(k),
// all k-points of the job in every launch.  Orthogonalising the columns of
// a Hermitian positive definite S by rotations V gives S V = W = U D: the
// eigenvalues are the column norms of W, the eigenvectors the columns of V
// (accumulated alongside, orthonormal to rounding and accurate to
// eps/gap even for the tiny eigenvalues the projector removes).  A sweep is
// Np - 1 rounds of the round-robin (circle) ordering of Np columns (Np = N
// rounded up to even, a zero padding column); a round rotates Np/2 disjoint
// column pairs, one CTA per (k-point, pair), so a launch has no inter-CTA
// dependency and a round is one kernel launch.  Per pair: alpha = |w_p|^2,
// beta = |w_q|^2, gamma = w_p^H w_q by a block reduction; with
// e = conj(gamma)/|gamma|, zeta = (beta - alpha)/(2|gamma|),
// t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t:
//   w_p <- c w_p - s e w_q,   w_q <- s w_p + c e w_q,
// which makes the pair orthogonal (the 2 x 2 Hermitian Jacobi rotation).  The
// largest |gamma|/sqrt(alpha beta) of a sweep decides convergence on the host.
//
// Since the eigenvalues are taken in ascending order and R~ is a product over
// k, R~ removes the m lowest positions at every k-point, m the largest count
// of eigenvalues below eps_d; T(k) c = c - U_m (U_m^H c), U_m the m lowest
// eigenvectors of S(k).
#include <cuda_runtime.h>
#include <math.h>

#include "fp64_elem.cuh"
#include "rpa_internal.h"

namespace rpa {
namespace {

__device__ __forceinline__ void round_pair(int n, int r, int i, int& p, int& q) {
  if (i == 0) {
    p = 0;
    q = 1 + (r % (n - 1));
  } else {
    p = 1 + ((r + i) % (n - 1));
    q = 1 + ((r + n - 1 - i) % (n - 1));
  }
}

// W[k][j][mu] = S(k)[mu][j] = conj(S(k)[j][mu]) (S Hermitian), V[k] = I;
// padding columns j >= N are zero in both.
template <bool C>
__global__ void __launch_bounds__(256) proj_load_kernel(ProjPtrs P, int N, int Np, double* __restrict__ W,
                                                        double* __restrict__ V) {
  const int k = blockIdx.y, j = blockIdx.x;
  const double* S = P.S[k];
  double* w = W + ((size_t)k * Np + j) * N * (C ? 2 : 1);
  double* v = V + ((size_t)k * Np + j) * N * (C ? 2 : 1);
  for (int mu = threadIdx.x; mu < N; mu += blockDim.x) {
    Elem<C> e = j < N ? conj_e<C>(ld_elem<C>(S, (long)j * N + mu)) : zero_elem<C>();
    st_elem<C>(w, mu, e);
    Elem<C> one = zero_elem<C>();
    one.re = (mu == j) ? 1.0 : 0.0;
    st_elem<C>(v, mu, one);
  }
}

// x <- c x - s e y, y <- s x + c e y for element mu of columns x, y.
template <bool C>
__device__ __forceinline__ void rotate_pair(double* xc, double* yc, int mu, double c, double s, double er, double ei) {
  const Elem<C> x = ld_elem<C>(xc, mu), y = ld_elem<C>(yc, mu);
  Elem<C> xn, yn;
  if constexpr (C) {
    const double eyr = er * y.re - ei * y.im, eyi = er * y.im + ei * y.re;
    xn.re = c * x.re - s * eyr;
    xn.im = c * x.im - s * eyi;
    yn.re = s * x.re + c * eyr;
    yn.im = s * x.im + c * eyi;
  } else {
    xn.re = c * x.re - s * er * y.re;
    yn.re = s * x.re + c * er * y.re;
  }
  st_elem<C>(xc, mu, xn);
  st_elem<C>(yc, mu, yn);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One round r: CTA (pair i, k-point k) rotates columns (p, q) of W[k].
template <bool C>
__global__ void __launch_bounds__(256) jacobi_round_kernel(int N, int Np, int r, double* __restrict__ W,
                                                           double* __restrict__ V, double thresh,
                                                           unsigned long long* __restrict__ off_max) {
  __shared__ double red[8][4];
  __shared__ double rot[5];  // c, s, e (re, im), applied flag
  const int i = blockIdx.x, k = blockIdx.y;
  int p, q;
  round_pair(Np, r, i, p, q);
  double* wp = W + ((size_t)k * Np + p) * N * (C ? 2 : 1);
  double* wq = W + ((size_t)k * Np + q) * N * (C ? 2 : 1);
  double a = 0.0, b = 0.0, gr = 0.0, gi = 0.0;
  for (int mu = threadIdx.x; mu < N; mu += blockDim.x) {
    const Elem<C> x = ld_elem<C>(wp, mu), y = ld_elem<C>(wq, mu);
    if constexpr (C) {
      a = fma(x.re, x.re, fma(x.im, x.im, a));
      b = fma(y.re, y.re, fma(y.im, y.im, b));
      gr = fma(x.re, y.re, fma(x.im, y.im, gr));  // conj(x) y
      gi = fma(x.re, y.im, fma(-x.im, y.re, gi));
    } else {
      a = fma(x.re, x.re, a);
      b = fma(y.re, y.re, b);
      gr = fma(x.re, y.re, gr);
    }
  }
  a = warp_sum(a);
  b = warp_sum(b);
  gr = warp_sum(gr);
  gi = warp_sum(gi);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[wid][0] = a;
    red[wid][1] = b;
    red[wid][2] = gr;
    red[wid][3] = gi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = gr = gi = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[w][0];
      b += red[w][1];
      gr += red[w][2];
      gi += red[w][3];
    }
    const double g = sqrt(gr * gr + gi * gi);
    const double off = (a > 0.0 && b > 0.0) ? g / sqrt(a * b) : 0.0;
    atomicMax(off_max, (unsigned long long)__double_as_longlong(off));
    if (off > thresh) {
      const double zeta = (b - a) / (2.0 * g);
      const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      rot[0] = c;
      rot[1] = c * t;
      rot[2] = gr / g;  // e = conj(gamma) / |gamma|
      rot[3] = -gi / g;
      rot[4] = 1.0;
    } else {
      rot[4] = 0.0;
    }
  }
  __syncthreads();
  if (rot[4] == 0.0) return;
  const double c = rot[0], s = rot[1], er = rot[2], ei = rot[3];
  double* vp = V + ((size_t)k * Np + p) * N * (C ? 2 : 1);
  double* vq = V + ((size_t)k * Np + q) * N * (C ? 2 : 1);
  for (int mu = threadIdx.x; mu < N; mu += blockDim.x) {
    rotate_pair<C>(wp, wq, mu, c, s, er, ei);
    rotate_pair<C>(vp, vq, mu, c, s, er, ei);
  }
}

// Per k-point: eigenvalue of column j = |w_j|, ascending rank (ties by index),
// count below eps_d (into m by atomicMax); lam_sorted[k][rank] and
// by_rank[k][rank] = j for the N real columns.
template <bool C>
__global__ void __launch_bounds__(256) proj_rank_kernel(int N, int Np, const double* __restrict__ W, double eps_d,
                                                        double* __restrict__ lam_sorted, int* __restrict__ by_rank,
                                                        int* __restrict__ m) {
  extern __shared__ double lam[];
  const int k = blockIdx.x;
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    const double* w = W + ((size_t)k * Np + j) * N * (C ? 2 : 1);
    double s = 0.0;
    for (int mu = 0; mu < N; ++mu) {
      const Elem<C> x = ld_elem<C>(w, mu);
      s = fma(x.re, x.re, s);
      if constexpr (C) s = fma(x.im, x.im, s);
    }
    lam[j] = sqrt(s);
  }
  __syncthreads();
  int below = 0;
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    // the padding column (zero) is not an eigenvector of S
    if (j >= N) continue;
    int rank = 0;
    for (int l = 0; l < N; ++l) rank += (lam[l] < lam[j]) || (lam[l] == lam[j] && l < j);
    lam_sorted[(size_t)k * N + rank] = lam[j];
    by_rank[(size_t)k * N + rank] = j;
    below += lam[j] - eps_d < 0.0;
  }
  below = __reduce_add_sync(0xffffffffu, below);
  __shared__ int wsum[8];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = below;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    atomicMax(m, t);
  }
}

// X[k][r][n] = sum_mu conj(u_r[mu]) c[mu][n] for the r < m lowest
// eigenvectors u_r = V[k][by_rank[r]].
template <bool C>
__global__ void __launch_bounds__(256) proj_x_kernel(ProjPtrs P, int N, int Np, int n_mo, const double* __restrict__ V,
                                                     const int* __restrict__ by_rank, const int* __restrict__ m,
                                                     double* __restrict__ X) {
  const int r = blockIdx.x, k = blockIdx.y;
  if (r >= *m) return;
  const int j = by_rank[(size_t)k * N + r];
  if (j < 0 || j >= N) return;  // ranks are a permutation unless an eigenvalue is NaN
  const double* u = V + ((size_t)k * Np + j) * N * (C ? 2 : 1);
  const double* c = P.c[k];
  double* x = X + ((size_t)k * N + r) * n_mo * (C ? 2 : 1);
  for (int n = threadIdx.x; n < n_mo; n += blockDim.x) {
    Elem<C> acc = zero_elem<C>();
    for (int mu = 0; mu < N; ++mu) mac<C>(acc, conj_e<C>(ld_elem<C>(u, mu)), ld_elem<C>(c, (long)mu * n_mo + n));
    st_elem<C>(x, n, acc);
  }
}

// c~[mu][n] = c[mu][n] - sum_{r < m} u_r[mu] X[r][n]  (may run in place: X
// was formed from c before).
template <bool C>
__global__ void __launch_bounds__(256) proj_apply_kernel(ProjPtrs P, int N, int Np, int n_mo,
                                                         const double* __restrict__ V, const int* __restrict__ by_rank,
                                                         const int* __restrict__ m, const double* __restrict__ X) {
  const int mu = blockIdx.x, k = blockIdx.y;
  const int mm = *m;
  const double* c = P.c[k];
  double* out = P.out[k];
  for (int n = threadIdx.x; n < n_mo; n += blockDim.x) {
    Elem<C> v = ld_elem<C>(c, (long)mu * n_mo + n);
    for (int r = 0; r < mm; ++r) {
      const int j = by_rank[(size_t)k * N + r];
      if (j < 0 || j >= N) continue;
      Elem<C> u = ld_elem<C>(V + ((size_t)k * Np + j) * N * (C ? 2 : 1), mu);
      u.re = -u.re;
      if constexpr (C) u.im = -u.im;
      mac<C>(v, u, ld_elem<C>(X + ((size_t)k * N + r) * n_mo * (C ? 2 : 1), n));
    }
    st_elem<C>(out, (long)mu * n_mo + n, v);
  }
}

}  // namespace

cudaError_t launch_proj_load(int cplx, const ProjPtrs& P, int n_mat, int N, int Np, double* W, double* V,
                             cudaStream_t s) {
  const dim3 grid(Np, n_mat);
  if (cplx)
    proj_load_kernel<true><<<grid, 256, 0, s>>>(P, N, Np, W, V);
  else
    proj_load_kernel<false><<<grid, 256, 0, s>>>(P, N, Np, W, V);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_round(int cplx, int n_mat, int N, int Np, int r, double* W, double* V, double thresh,
                                unsigned long long* off_max, cudaStream_t s) {
  const dim3 grid(Np / 2, n_mat);
  if (cplx)
    jacobi_round_kernel<true><<<grid, 256, 0, s>>>(N, Np, r, W, V, thresh, off_max);
  else
    jacobi_round_kernel<false><<<grid, 256, 0, s>>>(N, Np, r, W, V, thresh, off_max);
  return cudaGetLastError();
}

cudaError_t launch_proj_finish(int cplx, const ProjPtrs& P, int n_mat, int N, int Np, int n_mo, const double* W,
                               const double* V, double eps_d, double* lam_sorted, int* by_rank, int* m, double* X,
                               cudaStream_t s) {
  const size_t sh = sizeof(double) * Np;
  if (sh > 48 * 1024) return cudaErrorInvalidValue;
  if (cplx) {
    proj_rank_kernel<true><<<n_mat, 256, sh, s>>>(N, Np, W, eps_d, lam_sorted, by_rank, m);
    proj_x_kernel<true><<<dim3(N, n_mat), 256, 0, s>>>(P, N, Np, n_mo, V, by_rank, m, X);
    proj_apply_kernel<true><<<dim3(N, n_mat), 256, 0, s>>>(P, N, Np, n_mo, V, by_rank, m, X);
  } else {
    proj_rank_kernel<false><<<n_mat, 256, sh, s>>>(N, Np, W, eps_d, lam_sorted, by_rank, m);
    proj_x_kernel<false><<<dim3(N, n_mat), 256, 0, s>>>(P, N, Np, n_mo, V, by_rank, m, X);
    proj_apply_kernel<false><<<dim3(N, n_mat), 256, 0, s>>>(P, N, Np, n_mo, V, by_rank, m, X);
  }
  return cudaGetLastError();
}

}  // namespace rpa
