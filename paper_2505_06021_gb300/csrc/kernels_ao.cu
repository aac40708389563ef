// AO -> MO transform of the density-fitting coefficients (Sec. 2.2) on GB300.
//
// Sec. 2.2 expands the product of two Bloch basis functions in fit functions
// on the same two atoms (PADF); in reciprocal space the coefficients of the
// pair (k, k+q) come from one k-dependent array per k-point,
// C_{nu mu alpha}(kappa) with alpha on the atom of mu:
//   B^{mu nu}_gamma = [gamma on atom(mu)] C_{nu mu gamma}(k+q)
//                   + [gamma on atom(nu)] conj(C_{mu nu gamma}(k)),
// and the coefficients of the orbital pair psi*_i(k) psi_a(k+q) are
//   C_{gamma,ia}(q,k) = sum_{mu nu} conj(c_{mu i}(k)) c_{nu a}(k+q) B^{mu nu}_gamma.
//
// Summing each PADF term over the basis function that is not on gamma's atom
// first gives one half-transform per k-point and MO set,
//   H(kappa)[s(mu, gamma)][n] = sum_nu C_{nu mu gamma}(kappa) c_{nu n}(kappa),
// (s(mu, gamma) the PADF column of the pair), after which each (q, k) pair is a
// contraction over the nb(A) basis functions of gamma's atom A only:
//   C_{gamma,ia} = sum_{mu on A} conj(c_{mu i}(k)) H_virt(k+q)[s(mu,gamma)][a]
//                + sum_{nu on A} c_{nu a}(k+q) conj(H_occ(k)[s(nu,gamma)][i]).
// Work per pair 2 nb n_aux n_occ n_virt complex multiply-adds instead of
// n_bas^2 n_aux n_occ n_virt for the direct double sum; the half-transforms
// are done once per k-point, not once per pair.
//
// Lattice form: the k-dependent arrays are the lattice sums of the cell-pair
// coefficients (Sec. 2.2), C(kappa) = sum_dR C^{0,dR} e^{2 pi i kappa.n},
// formed one k-point at a time by padf_k_kernel just before its
// half-transforms (HBM-bound: n_R real reads and one complex write per entry).
//
// The transform kernels are FP64 (DFMA): the result feeds the FP64 chi0 path directly
// and the split-precision path through its own 31-bit slicing.  GB300 issues
// about two DFMA per clock per SM, so the kernels are organised only to keep
// that pipe busy: a 32 x 32 output tile per CTA, 2 x 2 outputs per thread,
// operands staged through shared memory in K-steps of 16 with coalesced row
// loads, every complex multiply-add four DFMAs.
#include <cuda_runtime.h>

#include <algorithm>

#include "fp64_elem.cuh"
#include "rpa_internal.h"

namespace rpa {
namespace {

constexpr int AT = 32;  // output tile edge
constexpr int AK = 16;  // K-step

// acc[u][v] += sum_k A(k, ty + 16u) * B(k, tx + 16v) over k in [0, K);
// la / lb return the operand (zero outside the tile's valid range).
template <bool C, class LA, class LB>
__device__ __forceinline__ void tile_tn(int K, const LA& la, const LB& lb, Elem<C> (&acc)[2][2],
                                        Elem<C> (*As)[AT], Elem<C> (*Bs)[AT]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += AK) {
    for (int idx = tid; idx < AK * AT; idx += 256) {
      const int kk = idx / AT, r = idx % AT, k = k0 + kk;
      As[kk][r] = k < K ? la(k, r) : zero_elem<C>();
      Bs[kk][r] = k < K ? lb(k, r) : zero_elem<C>();
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < AK; ++kk) {
      const Elem<C> a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const Elem<C> b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      mac<C>(acc[0][0], a0, b0);
      mac<C>(acc[0][1], a0, b1);
      mac<C>(acc[1][0], a1, b0);
      mac<C>(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
}

// H[s][n] = sum_nu P[nu][s] c[nu][n0 + n] for s < S, n < ncols.
template <bool C>
__global__ void __launch_bounds__(256) ao_half_kernel(int n_bas, int S, int n_mo, const double* __restrict__ P,
                                                      const double* __restrict__ c, int n0, int ncols,
                                                      double* __restrict__ H, int n_tn) {
  __shared__ Elem<C> As[AK][AT];
  __shared__ Elem<C> Bs[AK][AT];
  const int ts = blockIdx.x / n_tn, tn = blockIdx.x % n_tn;
  const int s0 = ts * AT, c0 = tn * AT;
  Elem<C> acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) acc[u][v] = zero_elem<C>();
  auto la = [&](int k, int r) {
    return s0 + r < S ? ld_elem<C>(P, (long)k * S + s0 + r) : zero_elem<C>();
  };
  auto lb = [&](int k, int r) {
    return c0 + r < ncols ? ld_elem<C>(c, (long)k * n_mo + n0 + c0 + r) : zero_elem<C>();
  };
  tile_tn<C>(n_bas, la, lb, acc, As, Bs);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int s = s0 + ty + 16 * u, n = c0 + tx + 16 * v;
      if (s < S && n < ncols) st_elem<C>(H, (long)s * ncols + n, acc[u][v]);
    }
}

// One CTA: fit function gamma of pair p, a 32 x 32 tile of (i, a).
template <bool C>
__global__ void __launch_bounds__(256)
    ao_assemble_kernel(const __grid_constant__ AoPairs pr, const int4* __restrict__ fit, int n_aux, int n_occ,
                       int n_virt, int n_mo, int n_ti, int n_ta) {
  __shared__ Elem<C> As[AK][AT];
  __shared__ Elem<C> Bs[AK][AT];
  long bid = blockIdx.x;
  const int ta = (int)(bid % n_ta);
  bid /= n_ta;
  const int ti = (int)(bid % n_ti);
  bid /= n_ti;
  const int gamma = (int)(bid % n_aux);
  const int p = (int)(bid / n_aux);
  const int4 f = fit[gamma];  // first basis function of gamma's atom, its count, H row of (0, gamma), fit count
  const int b0 = f.x, nb = f.y, row0 = f.z, nf = f.w;
  const int i0 = ti * AT, a0 = ta * AT;
  const double* ck = pr.mo_k[p];
  const double* ckq = pr.mo_kq[p];
  const double* Hk = pr.h_occ[p];
  const double* Hkq = pr.h_virt[p];
  Elem<C> acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) acc[u][v] = zero_elem<C>();
  // k < nb: conj(c_{mu i}(k)) * H_virt(k+q)[s(mu, gamma)][a], mu = b0 + k
  // k >= nb: conj(H_occ(k)[s(nu, gamma)][i]) * c_{nu a}(k+q), nu = b0 + k - nb
  auto la = [&](int k, int r) {
    const int i = i0 + r;
    if (i >= n_occ) return zero_elem<C>();
    return k < nb ? conj_e<C>(ld_elem<C>(ck, (long)(b0 + k) * n_mo + i))
                  : conj_e<C>(ld_elem<C>(Hk, (long)(row0 + (long)(k - nb) * nf) * n_occ + i));
  };
  auto lb = [&](int k, int r) {
    const int a = a0 + r;
    if (a >= n_virt) return zero_elem<C>();
    return k < nb ? ld_elem<C>(Hkq, (long)(row0 + (long)k * nf) * n_virt + a)
                  : ld_elem<C>(ckq, (long)(b0 + k - nb) * n_mo + n_occ + a);
  };
  tile_tn<C>(2 * nb, la, lb, acc, As, Bs);
  double* out = pr.out[p] + (size_t)gamma * n_occ * n_virt * (C ? 2 : 1);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + ty + 16 * u, a = a0 + tx + 16 * v;
      if (i < n_occ && a < n_virt) st_elem<C>(out, (long)i * n_virt + a, acc[u][v]);
    }
}

// out[e] = sum_r C0[r][e] e^{2 pi i kappa . R_r}; real jobs keep the real part
// (Gamma-equivalent k-points only, where every phase is 1).
template <bool C>
__global__ void __launch_bounds__(256) padf_k_kernel(const __grid_constant__ PadfLattice L, double k0, double k1,
                                                     double k2, long n, double* __restrict__ out) {
  __shared__ double cs[PadfLattice::kMax], sn[PadfLattice::kMax];
  for (int r = threadIdx.x; r < L.n_R; r += blockDim.x) {
    const double x = k0 * L.R[r][0] + k1 * L.R[r][1] + k2 * L.R[r][2];
    sincospi(2.0 * x, &sn[r], &cs[r]);
  }
  __syncthreads();
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int r = 0; r < L.n_R; ++r) {
      const double v = __ldcs(L.C0[r] + e);
      re = fma(v, cs[r], re);
      if constexpr (C) im = fma(v, sn[r], im);
    }
    if constexpr (C)
      *reinterpret_cast<double2*>(out + 2 * e) = make_double2(re, im);
    else
      out[e] = re;
  }
}

}  // namespace

cudaError_t launch_padf_k(int cplx, const PadfLattice& L, const double* kfrac, long n, double* out,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (L.n_R <= 0 || L.n_R > PadfLattice::kMax) return cudaErrorInvalidValue;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long blocks = std::min<long>((n + 255) / 256, (long)sms * 16);
  if (cplx)
    padf_k_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(L, kfrac[0], kfrac[1], kfrac[2], n, out);
  else
    padf_k_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(L, kfrac[0], kfrac[1], kfrac[2], n, out);
  return cudaGetLastError();
}

cudaError_t launch_ao_half(int cplx, int n_bas, int S, int n_mo, const double* P, const double* c, int n0, int ncols,
                           double* H, cudaStream_t s) {
  if (S <= 0 || ncols <= 0) return cudaSuccess;
  const int n_ts = (S + AT - 1) / AT, n_tn = (ncols + AT - 1) / AT;
  const long blocks = (long)n_ts * n_tn;
  if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
  if (cplx)
    ao_half_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(n_bas, S, n_mo, P, c, n0, ncols, H, n_tn);
  else
    ao_half_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(n_bas, S, n_mo, P, c, n0, ncols, H, n_tn);
  return cudaGetLastError();
}

cudaError_t launch_ao_assemble(int cplx, const AoPairs& pr, int n_pairs, const int4* fit, int n_aux, int n_occ,
                               int n_virt, int n_mo, cudaStream_t s) {
  if (n_pairs <= 0) return cudaSuccess;
  if (n_pairs > AoPairs::kMax) return cudaErrorInvalidValue;
  const int n_ti = (n_occ + AT - 1) / AT, n_ta = (n_virt + AT - 1) / AT;
  const long blocks = (long)n_pairs * n_aux * n_ti * n_ta;
  if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
  if (cplx)
    ao_assemble_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(pr, fit, n_aux, n_occ, n_virt, n_mo, n_ti, n_ta);
  else
    ao_assemble_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(pr, fit, n_aux, n_occ, n_virt, n_mo, n_ti, n_ta);
  return cudaGetLastError();
}

}  // namespace rpa
