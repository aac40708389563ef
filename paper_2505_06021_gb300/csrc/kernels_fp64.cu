// FP64 kernels of the RPA hot path on GB300 (sm_103a).
//
// GB300 executes FP64 at about 1/58 of its FP32 rate (1.2 TFLOP/s measured
// for DFMA and DGEMM), so every kernel here is bound by the FP64 pipe and is
// organised to issue as few FP64 instructions per useful result as possible:
//   * chi0: the product conj(C_P,t) C_Q,t is formed once per t and reused for
//     a group of G frequencies (2 DFMA per frequency instead of 4), and only
//     the lower triangle of tiles is computed (chi0 is Hermitian);
//   * the sandwich uses the Cholesky factor L of V (triangular operands, lower
//     output only) instead of the dense V^(1/2);
//   * the factorisation of 1 - Pi keeps the diagonal in "pivot minus one"
//     form so that ln det = sum log1p(u) keeps its digits as Pi -> 0;
//   * the inverse form used with the split-precision chi0 needs no sandwich at
//     all: det(1 - V^(1/2) chi V^(1/2)) = det(V^-1 - chi) det V and
//     Tr(V^(1/2) chi V^(1/2)) = Tr(chi V), with V^-1 = X^H X, X = L^-1, formed
//     once per q.
// All reductions run in a fixed order, so results are bit-reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "fp64_elem.cuh"
#include "rpa_internal.h"

namespace rpa {
namespace {

// ---------------------------------------------------------------- helpers --

int num_sms_fp64() { return device_sm_count(); }

// Lower-triangular tile index -> (I, J), J <= I.
__device__ __forceinline__ void tri_index(int t, int& I, int& J) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// ------------------------------------------------------------ d table -----

__global__ void dtab_kernel(BatchGeom g, const double* __restrict__ eps_occ, const double* __restrict__ eps_virt,
                            const int* __restrict__ kidx, const int* __restrict__ kqidx,
                            const double* __restrict__ omega, double zeta_k, double* __restrict__ dtab) {
  const long total = (long)g.n_qb * g.n_k * g.n_w * g.n_ov;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    long r = idx;
    const int t = (int)(r % g.n_ov);
    r /= g.n_ov;
    const int w = (int)(r % g.n_w);
    r /= g.n_w;
    const int pair = (int)r;  // qb * n_k + j
    const int i = t / g.n_virt, a = t - i * g.n_virt;
    const double delta = eps_virt[(long)kqidx[pair] * g.n_virt + a] - eps_occ[(long)kidx[pair] * g.n_occ + i];
    const double om = omega[w];
    dtab[idx] = zeta_k * (-4.0 * delta / (delta * delta + om * om));
  }
}

// --------------------------------------------------------------- chi0 -----
// Grid: one CTA per (q in batch, lower tile pair (I, J), frequency group).
// Tile 32 x 32 outputs, 256 threads, each thread a 2 x 2 block of outputs
// (rows ty, ty+16; columns tx, tx+16) for G frequencies.

constexpr int CT = 32;  // output tile edge
constexpr int TK = 16;  // t-chunk

template <bool C, int G>
__global__ void __launch_bounds__(256, 1)
    chi0_fp64_kernel(BatchGeom g, const double* const* __restrict__ Cptrs, const double* __restrict__ dtab,
                     double* __restrict__ chi, int n_tiles, int n_wg) {
  __shared__ Elem<C> As[TK][CT];
  __shared__ Elem<C> Bs[TK][CT];
  __shared__ double Ds[G][TK];

  int bid = blockIdx.x;
  const int wg = bid % n_wg;
  bid /= n_wg;
  const int tile = bid % n_tiles;
  const int qb = bid / n_tiles;
  int I, J;
  tri_index(tile, I, J);
  const int w0 = wg * G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int N = g.n_aux, n_ov = g.n_ov;

  Elem<C> acc[G][4];
#pragma unroll
  for (int k = 0; k < G; ++k)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[k][m] = zero_elem<C>();

  for (int j = 0; j < g.n_k; ++j) {
    const double* Cj = Cptrs[qb * g.n_k + j];
    const double* dj = dtab + ((long)(qb * g.n_k + j) * g.n_w) * n_ov;
    for (int t0 = 0; t0 < n_ov; t0 += TK) {
      for (int idx = tid; idx < CT * TK; idx += 256) {
        const int r = idx / TK, tt = idx % TK, t = t0 + tt;
        const int P = I * CT + r, Q = J * CT + r;
        As[tt][r] = (P < N && t < n_ov) ? ld_elem<C>(Cj, (long)P * n_ov + t) : zero_elem<C>();
        Bs[tt][r] = (Q < N && t < n_ov) ? ld_elem<C>(Cj, (long)Q * n_ov + t) : zero_elem<C>();
      }
      for (int idx = tid; idx < G * TK; idx += 256) {
        const int k = idx / TK, tt = idx % TK, t = t0 + tt, w = w0 + k;
        Ds[k][tt] = (t < n_ov && w < g.n_w) ? dj[(long)w * n_ov + t] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int tt = 0; tt < TK; ++tt) {
        const Elem<C> a0 = As[tt][ty], a1 = As[tt][ty + 16];
        const Elem<C> b0 = Bs[tt][tx], b1 = Bs[tt][tx + 16];
        // p = conj(a) * b
        Elem<C> p[4];
        const Elem<C> aa[2] = {a0, a1}, bb[2] = {b0, b1};
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            if constexpr (C) {
              p[2 * u + v].re = fma(aa[u].re, bb[v].re, aa[u].im * bb[v].im);
              p[2 * u + v].im = fma(aa[u].re, bb[v].im, -aa[u].im * bb[v].re);
            } else {
              p[2 * u + v].re = aa[u].re * bb[v].re;
            }
          }
#pragma unroll
        for (int k = 0; k < G; ++k) {
          const double d = Ds[k][tt];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            acc[k][m].re = fma(d, p[m].re, acc[k][m].re);
            if constexpr (C) acc[k][m].im = fma(d, p[m].im, acc[k][m].im);
          }
        }
      }
      __syncthreads();
    }
  }
  // write the lower triangle and its Hermitian mirror
  const long NN = (long)N * N;
#pragma unroll
  for (int k = 0; k < G; ++k) {
    const int w = w0 + k;
    if (w >= g.n_w) break;
    double* out = chi + ((long)qb * g.n_w + w) * NN * (C ? 2 : 1);
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int P = I * CT + ty + 16 * u, Q = J * CT + tx + 16 * v;
        if (P >= N || Q >= N || Q > P) continue;
        Elem<C> e = acc[k][2 * u + v];
        if (P == Q) {
          if constexpr (C) e.im = 0.0;
          st_elem<C>(out, (long)P * N + Q, e);
        } else {
          st_elem<C>(out, (long)P * N + Q, e);
          st_elem<C>(out, (long)Q * N + P, conj_e<C>(e));
        }
      }
  }
}

template <bool C, int G>
cudaError_t chi0_launch_g(const BatchGeom& g, const double* const* Cptrs, const double* dtab, double* chi,
                          cudaStream_t s) {
  const int nt = (g.n_aux + CT - 1) / CT;
  const int n_tiles = nt * (nt + 1) / 2;
  const int n_wg = (g.n_w + G - 1) / G;
  const long blocks = (long)n_tiles * n_wg * g.n_qb;
  if (blocks > 0x7fffffffL) return cudaErrorInvalidConfiguration;
  chi0_fp64_kernel<C, G><<<(unsigned)blocks, 256, 0, s>>>(g, Cptrs, dtab, chi, n_tiles, n_wg);
  return cudaGetLastError();
}

// Frequency group size: minimises FP64 instructions per (P, Q, t),
// 4 * ceil(n_w / G) (products, complex) + 2 * G * ceil(n_w / G) (weights).
int pick_group(int n_w) {
  const int cand[4] = {4, 5, 8, 10};
  int best = 8;
  long best_cost = -1;
  for (int c : cand) {
    const long ng = (n_w + c - 1) / c;
    const long cost = 4 * ng + 2 * (long)c * ng;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

template <bool C>
cudaError_t chi0_dispatch(const BatchGeom& g, const double* const* Cptrs, const double* dtab, double* chi,
                          cudaStream_t s) {
  switch (pick_group(g.n_w)) {
    case 4:
      return chi0_launch_g<C, 4>(g, Cptrs, dtab, chi, s);
    case 5:
      return chi0_launch_g<C, 5>(g, Cptrs, dtab, chi, s);
    case 10:
      return chi0_launch_g<C, 10>(g, Cptrs, dtab, chi, s);
    default:
      return chi0_launch_g<C, 8>(g, Cptrs, dtab, chi, s);
  }
}

// ----------------------------------------------------------- sandwich -----
// MODE 0: T = X L      (L lower triangular; K-range of output column tile J
//                       starts at J*64)
// MODE 1: Y = -L^H T   (lower output tiles only; K-range of row tile I starts
//                       at I*64)
// 64 x 64 output tile, 256 threads, 4 x 4 outputs per thread.

constexpr int GT = 64;
constexpr int GK = 16;

template <bool C, int MODE>
__global__ void __launch_bounds__(256)
    sandwich_kernel(int N, int n_w, const double* __restrict__ Xb, const double* __restrict__ Lb,
                    double* __restrict__ Ob, int n_tiles_row, int tiles_per_mat) {
  __shared__ Elem<C> As[GK][GT];
  __shared__ Elem<C> Bs[GK][GT];
  const int b = blockIdx.x / tiles_per_mat;
  const int tile = blockIdx.x % tiles_per_mat;
  int I, J;
  if (MODE == 0) {
    I = tile / n_tiles_row;
    J = tile % n_tiles_row;
  } else {
    tri_index(tile, I, J);
  }
  const long NN = (long)N * N;
  const int cs = C ? 2 : 1;
  const double* X = Xb + (long)b * NN * cs;
  const double* L = Lb + (long)(b / n_w) * NN * cs;
  double* O = Ob + (long)b * NN * cs;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  Elem<C> acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = zero_elem<C>();

  const int k_begin = (MODE == 0 ? J : I) * GT;
  for (int k0 = k_begin; k0 < N; k0 += GK) {
    for (int idx = tid; idx < GK * GT; idx += 256) {
      if (MODE == 0) {
        // A = X[P][R] (row-major, R contiguous): idx -> (p, kk) with kk fastest
        const int p = idx / GK, kk = idx % GK, P = I * GT + p, R = k0 + kk;
        As[kk][p] = (P < N && R < N) ? ld_elem<C>(X, (long)P * N + R) : zero_elem<C>();
        // B = L[R][Q], zero above the diagonal (R < Q)
        const int q = idx % GT, kb = idx / GT, Q = J * GT + q, R2 = k0 + kb;
        Bs[kb][q] = (Q < N && R2 < N && R2 >= Q) ? ld_elem<C>(L, (long)R2 * N + Q) : zero_elem<C>();
      } else {
        // A[P][R] = conj(L[R][P]), zero for R < P; read L rows R, P contiguous
        const int p = idx % GT, kk = idx / GT, P = I * GT + p, R = k0 + kk;
        As[kk][p] = (P < N && R < N && R >= P) ? conj_e<C>(ld_elem<C>(L, (long)R * N + P)) : zero_elem<C>();
        const int q = idx % GT, Q = J * GT + q;
        Bs[kk][q] = (Q < N && R < N) ? ld_elem<C>(X, (long)R * N + Q) : zero_elem<C>();
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      Elem<C> a[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = Bs[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) mac<C>(acc[u][v], a[u], bv[v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int P = I * GT + ty + 16 * u, Q = J * GT + tx + 16 * v;
      if (P >= N || Q >= N) continue;
      Elem<C> e = acc[u][v];
      if (MODE == 1) {
        e.re = -e.re;
        if constexpr (C) e.im = -e.im;
      }
      st_elem<C>(O, (long)P * N + Q, e);
    }
}

// ----------------------------------------------------------- Cholesky -----
// One CTA (256 threads) per matrix, right-looking blocked with 32-wide panels.
// mode 0: A holds Y = -Pi; the factorised matrix is 1 + Y, whose diagonal is
//         kept as u = pivot - 1; ln det = sum_j log1p(u_j); Tr Pi = -sum Y_jj.
// mode 1: A holds V; factor in place, strict upper triangle zeroed; with out
//         set, out[b] = ln det V.
// mode 2 (inverse form): A holds chi of (q, w) = (b / n_w, b % n_w); the
//         lower triangle becomes M = V^-1 - chi (Wn = -V^-1 of the q, lower
//         triangle), factorised; ln det(1 - Pi) = ln det M + ln det V
//         (ldV[q]) and Tr Pi = Tr(chi V) = sum_PQ Re(chi_PQ conj(V_PQ)) from
//         the copy Vc of V(q).

constexpr int CB = 32;

// Synchronisation and shared-memory access across the CTAs that share one
// matrix: a thread-block cluster of CL CTAs (CL = 1: a single CTA).
template <int CL>
struct Team {
  __device__ static unsigned rank() {
    if constexpr (CL == 1) {
      return 0;
    } else {
      unsigned r;
      asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
      return r;
    }
  }
  __device__ static void sync() {
    if constexpr (CL == 1) {
      __syncthreads();
    } else {
      __syncthreads();
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
  }
  // value of a shared variable in CTA `r` of the team
  template <typename T>
  __device__ static T read(T* p, unsigned r) {
    if constexpr (CL == 1) {
      return *p;
    } else {
      const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p));
      uint32_t remote;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
      T v;
      if constexpr (sizeof(T) == 8) {
        unsigned long long x;
        asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(x) : "r"(remote) : "memory");
        memcpy(&v, &x, 8);
      } else {
        unsigned x;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(x) : "r"(remote) : "memory");
        memcpy(&v, &x, 4);
      }
      return v;
    }
  }
};

// Matrix loads go to L2 (ld.global.cg): each element is read once per panel
// step, so L1 gains nothing, and in the cluster variant other CTAs write the
// matrix between the barriers.
template <bool C, int CL>
__device__ __forceinline__ Elem<C> ldm(const double* p, long i) {
  Elem<C> e;
  if constexpr (C) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p + 2 * i));
    e.re = v.x;
    e.im = v.y;
  } else {
    e.re = __ldcg(p + i);
  }
  return e;
}

// Fixed-order sum of the per-thread values `s` over the whole team; the
// result is valid in every thread of CTA 0 (red[0]).
template <int CL>
__device__ void team_sum(double s, double* red, double* part) {
  const int tid = threadIdx.x;
  red[tid] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (tid < off) red[tid] += red[tid + off];
    __syncthreads();
  }
  if (tid == 0) *part = red[0];
  Team<CL>::sync();
  if (Team<CL>::rank() == 0 && tid == 0) {
    double t = 0.0;
    for (unsigned r = 0; r < (unsigned)CL; ++r) t += Team<CL>::read(part, r);
    red[0] = t;
  }
  __syncthreads();
}

// Right-looking blocked Cholesky with 32-wide panels.  One matrix per team of
// CL CTAs (256 threads each): CTA 0 factors the diagonal block, the panel rows
// and the trailing tiles are dealt round robin over the team, barriers between
// the phases.  Sums that enter the results (trace, log-det) run in a fixed
// order, so the value does not depend on CL's scheduling.
// mode 0: A holds Y = -Pi; the factorised matrix is 1 + Y, whose diagonal is
//         kept as u = pivot - 1; ln det = sum_j log1p(u_j); Tr Pi = -sum Y_jj.
// mode 1: A holds V; factor in place, strict upper triangle zeroed; with out
//         set, out[b] = ln det V.
// mode 2 (inverse form): A holds chi of (q, w) = (b / n_w, b % n_w); the
//         lower triangle becomes M = V^-1 - chi (Wn = -V^-1 of the q, lower
//         triangle), factorised; ln det(1 - Pi) = ln det M + ln det V
//         (ldV[q]) and Tr Pi = Tr(chi V) = sum_PQ Re(chi_PQ conj(V_PQ)) from
//         the copy Vc of V(q).  The strict upper triangle (chi's redundant
//         half) is overwritten by float-float copies of the panels.
// One matrix A (N x N) in `mode`; out: 1 double (mode 1) or 2 (ln det, Tr);
// on a non-positive pivot *status becomes `code` (if still 0).  Mode 2 reads
// Wq = -V^-1 and Vq = V of the matrix's q and ldv = ln det V.
template <bool C, int CL>
__device__ __forceinline__ void chol_one(int N, double* __restrict__ A, int mode, double* __restrict__ out,
                                         int* __restrict__ status, int code, const double* __restrict__ Wq,
                                         const double* __restrict__ Vq, const double* __restrict__ ldv) {
  __shared__ Elem<C> D[CB][CB + 1];
  __shared__ Elem<C> S2[CB][CB + 1];
  Elem<C>(*S1)[CB + 1] = D;  // the diagonal block is free again during the trailing update
  __shared__ double red[256];
  __shared__ double part;
  __shared__ int bad;
  __shared__ double logacc;
  const unsigned rank = Team<CL>::rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gtid = (int)rank * 256 + tid;
  constexpr int GSTRIDE = 256 * CL;

  // trace of Pi (modes 0 and 2); mode 2 also forms M in the lower triangle
  if (mode == 0) {
    double s = 0.0;
    for (int j = gtid; j < N; j += GSTRIDE) s += ldm<C, CL>(A, (long)j * N + j).re;
    team_sum<CL>(s, red, &part);
  } else if (mode == 2) {
    const long NN = (long)N * N;
    double s = 0.0;
    for (long idx = gtid; idx < NN; idx += GSTRIDE) {
      const int r = (int)(idx / N), c = (int)(idx % N);
      if (c > r) continue;
      const Elem<C> x = ldm<C, CL>(A, idx), v = ld_elem<C>(Vq, idx), w = ld_elem<C>(Wq, idx);
      double t = x.re * v.re;
      if constexpr (C) t = fma(x.im, v.im, t);
      s += (r == c) ? t : 2.0 * t;
      Elem<C> m;
      m.re = -w.re - x.re;
      if constexpr (C) m.im = -w.im - x.im;
      st_elem<C>(A, idx, m);
    }
    team_sum<CL>(s, red, &part);
  }
  if (tid == 0) {
    bad = 0;
    logacc = 0.0;
  }
  Team<CL>::sync();

  bool failed = false;
  for (int kb = 0; kb < N; kb += CB) {
    const int nb = min(CB, N - kb);
    // (i) diagonal block, by CTA 0
    if (rank == 0) {
      for (int idx = tid; idx < CB * CB; idx += 256) {
        const int r = idx / CB, c = idx % CB;
        D[r][c] = (r < nb && c <= r) ? ldm<C, CL>(A, (long)(kb + r) * N + kb + c) : zero_elem<C>();
      }
      __syncthreads();
      if (warp == 0) {
        double lacc = 0.0;
        int lbad = 0;
        for (int c = 0; c < nb; ++c) {
          double l = 0.0;
          if (lane == c) {
            const double u = D[c][c].re;
            const double piv = (mode == 0) ? 1.0 + u : u;
            if (!(piv > 0.0)) {
              lbad = 1;
            } else {
              l = sqrt(piv);
              lacc += (mode == 0) ? log1p(u) : log(piv);
              Elem<C> e = zero_elem<C>();
              e.re = l;
              D[c][c] = e;
            }
          }
          const int anybad = __any_sync(0xffffffffu, lbad);
          if (anybad) {
            lbad = 1;
            break;
          }
          l = __shfl_sync(0xffffffffu, l, c);
          __syncwarp();
          if (lane > c && lane < nb) {
            Elem<C> e = D[lane][c];
            e.re /= l;
            if constexpr (C) e.im /= l;
            D[lane][c] = e;
          }
          __syncwarp();
          if (lane > c && lane < nb) {
            const Elem<C> lr = D[lane][c];
            for (int cc = c + 1; cc <= lane; ++cc) {
              const Elem<C> lc = conj_e<C>(D[cc][c]);
              Elem<C> e = D[lane][cc];
              Elem<C> prod = zero_elem<C>();
              mac<C>(prod, lr, lc);
              e.re -= prod.re;
              if constexpr (C) e.im -= prod.im;
              D[lane][cc] = e;
            }
          }
          __syncwarp();
        }
        // lane-wise partial log sums, combined in lane order (fixed)
        for (int l2 = 0; l2 < 32; ++l2) {
          const double v = __shfl_sync(0xffffffffu, lacc, l2);
          if (lane == 0) logacc += v;
        }
        if (lbad && lane == 0) bad = 1;
      }
      __syncthreads();
      if (!bad) {
        for (int idx = tid; idx < CB * CB; idx += 256) {
          const int r = idx / CB, c = idx % CB;
          if (r < nb && c <= r) st_elem<C>(A, (long)(kb + r) * N + kb + c, D[r][c]);
        }
      }
    }
    Team<CL>::sync();
    if (Team<CL>::read(&bad, 0u)) {
      failed = true;
      break;
    }
    // (ii) panel: rows i >= kb + nb solve X L_kk^H = A_panel
    if (rank != 0) {
      for (int idx = tid; idx < CB * CB; idx += 256) {
        const int r = idx / CB, c = idx % CB;
        D[r][c] = (r < nb && c <= r) ? ldm<C, CL>(A, (long)(kb + r) * N + kb + c) : zero_elem<C>();
      }
      __syncthreads();
    }
    for (int i = kb + nb + gtid; i < N; i += GSTRIDE) {
      Elem<C> x[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        if (c < nb) {
          Elem<C> v = ldm<C, CL>(A, (long)i * N + kb + c);
#pragma unroll
          for (int c2 = 0; c2 < CB; ++c2) {
            if (c2 < c) {
              Elem<C> prod = zero_elem<C>();
              mac<C>(prod, x[c2], conj_e<C>(D[c][c2]));
              v.re -= prod.re;
              if constexpr (C) v.im -= prod.im;
            }
          }
          const double dd = D[c][c].re;
          v.re /= dd;
          if constexpr (C) v.im /= dd;
          x[c] = v;
          st_elem<C>(A, (long)i * N + kb + c, v);
          // mode 2: the float-float copy of L_{i,kb+c} for the trailing
          // update, converted once here instead of once per tile that reads
          // it; it goes to the free strict upper triangle (row kb + c, column
          // i > kb + c), so a tile's operand rows are contiguous there
          if (mode == 2) st_ff<C>(A, (long)(kb + c) * N + i, to_ff<C>(v));
        }
      }
    }
    Team<CL>::sync();
    // (iii) trailing update of the lower part of A[kb+nb:, kb+nb:]
    const int m0 = kb + nb;
    const int m = N - m0;
    if (m > 0 && mode == 2) {
      // inverse form (split-precision path): the update in float-float on the
      // FP32 pipe, about 2^-46 relative per product, five times the rate of
      // the FP64 pipe; the diagonal block and the panel stay FP64
      FFE<C>(*F1)[CB + 1] = reinterpret_cast<FFE<C>(*)[CB + 1]>(S1);
      FFE<C>(*F2)[CB + 1] = reinterpret_cast<FFE<C>(*)[CB + 1]>(S2);
      const int nt = (m + CB - 1) / CB;
      const int ntiles = nt * (nt + 1) / 2;
      const int tx = tid & 15, ty = tid >> 4;
      for (int tt = (int)rank; tt < ntiles; tt += CL) {
        int TI, TJ;
        tri_index(tt, TI, TJ);
        for (int idx = tid; idx < CB * CB; idx += 256) {
          const int r = idx % CB, c = idx / CB;
          const int ri = m0 + TI * CB + r, rj = m0 + TJ * CB + r;
          const long up = (long)(kb + c) * N;
          F1[c][r] = (ri < N && c < nb) ? ld_ff<C>(A, up + ri) : FFE<C>{};
          F2[c][r] = (rj < N && c < nb) ? conj_ff<C>(ld_ff<C>(A, up + rj)) : FFE<C>{};
        }
        __syncthreads();
        FFE<C> acc[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) acc[u][v] = to_ff<C>(zero_elem<C>());
        for (int c = 0; c < nb; ++c) {
          const FFE<C> a0 = F1[c][ty], a1 = F1[c][ty + 16];
          const FFE<C> b0 = F2[c][tx], b1 = F2[c][tx + 16];
          ff_mac_e<C>(acc[0][0], a0, b0);
          ff_mac_e<C>(acc[0][1], a0, b1);
          ff_mac_e<C>(acc[1][0], a1, b0);
          ff_mac_e<C>(acc[1][1], a1, b1);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int r = m0 + TI * CB + ty + 16 * u, c = m0 + TJ * CB + tx + 16 * v;
            if (r < N && c <= r) {
              Elem<C> e = ldm<C, CL>(A, (long)r * N + c);
              e.re -= (double)acc[u][v].rh + (double)acc[u][v].rl;
              if constexpr (C) e.im -= (double)acc[u][v].ih + (double)acc[u][v].il;
              st_elem<C>(A, (long)r * N + c, e);
            }
          }
        __syncthreads();
      }
    } else if (m > 0) {
      const int nt = (m + CB - 1) / CB;
      const int ntiles = nt * (nt + 1) / 2;
      const int tx = tid & 15, ty = tid >> 4;
      for (int tt = (int)rank; tt < ntiles; tt += CL) {
        int TI, TJ;
        tri_index(tt, TI, TJ);
        for (int idx = tid; idx < CB * CB; idx += 256) {
          const int r = idx / CB, c = idx % CB;
          const int ri = m0 + TI * CB + r, rj = m0 + TJ * CB + r;
          S1[c][r] = (ri < N && c < nb) ? ldm<C, CL>(A, (long)ri * N + kb + c) : zero_elem<C>();
          S2[c][r] = (rj < N && c < nb) ? conj_e<C>(ldm<C, CL>(A, (long)rj * N + kb + c)) : zero_elem<C>();
        }
        __syncthreads();
        Elem<C> acc[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) acc[u][v] = zero_elem<C>();
        for (int c = 0; c < nb; ++c) {
          const Elem<C> a0 = S1[c][ty], a1 = S1[c][ty + 16];
          const Elem<C> b0 = S2[c][tx], b1 = S2[c][tx + 16];
          mac<C>(acc[0][0], a0, b0);
          mac<C>(acc[0][1], a0, b1);
          mac<C>(acc[1][0], a1, b0);
          mac<C>(acc[1][1], a1, b1);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int r = m0 + TI * CB + ty + 16 * u, c = m0 + TJ * CB + tx + 16 * v;
            if (r < N && c <= r) {
              Elem<C> e = ldm<C, CL>(A, (long)r * N + c);
              e.re -= acc[u][v].re;
              if constexpr (C) e.im -= acc[u][v].im;
              st_elem<C>(A, (long)r * N + c, e);
            }
          }
        __syncthreads();
      }
    }
    Team<CL>::sync();
  }
  if (failed) {
    if (rank == 0 && tid == 0) {
      if (status) atomicCAS(status, 0, code);
      if (out) {
        out[0] = nan("");
        if (mode != 1) out[1] = nan("");
      }
    }
  } else {
    if (mode == 1) {
      for (long idx = gtid; idx < (long)N * N; idx += GSTRIDE) {
        const int r = (int)(idx / N), c = (int)(idx % N);
        if (c > r) st_elem<C>(A, idx, zero_elem<C>());
      }
    }
    if (rank == 0 && tid == 0 && out) {
      if (mode == 0) {
        out[0] = logacc;
        out[1] = -red[0];
      } else if (mode == 2) {
        out[0] = logacc + *ldv;
        out[1] = red[0];
      } else {
        out[0] = logacc;
      }
    }
  }
  // no CTA leaves while another may still read its shared memory
  Team<CL>::sync();
}

// One-CTA-per-matrix Cholesky launches keep two matrices on each SM (128
// registers per thread): while one CTA is in its serial phases (the diagonal
// block in one warp, the panel solve, barriers) the other keeps the FP64 pipe
// busy with its trailing update.
constexpr int CHOL_CTAS_PER_SM = 2;

// Batched: matrix b of the launch (team b / CL) at mats + b * bstride.
template <bool C, int CL>
__global__ void __launch_bounds__(256, CL == 1 ? CHOL_CTAS_PER_SM : 1)
    cholesky_kernel(int N, double* __restrict__ mats, long bstride, int mode, double* __restrict__ out,
                    int* __restrict__ status, int status_base, const double* __restrict__ Wn,
                    const double* __restrict__ Vc, const double* __restrict__ ldV, int n_w, int b0) {
  const int b = b0 + (int)(blockIdx.x / CL);
  const long q = mode == 2 ? b / n_w : 0;
  const long NN = (long)N * N * (C ? 2 : 1);
  chol_one<C, CL>(N, mats + (long)b * bstride, mode, out ? out + (mode == 1 ? b : 2 * b) : nullptr, status,
                  1 + status_base + b, mode == 2 ? Wn + q * NN : nullptr, mode == 2 ? Vc + q * NN : nullptr,
                  mode == 2 ? ldV + q : nullptr);
}

// Ragged: one CTA per task, matrices of any size (tasks ordered largest
// first by the caller, so the block scheduler packs them greedily).
// (One CTA per SM: with uneven sizes the second CTA's register cap costs more
// than the overlap gains; measured on the batched workload.)
template <bool C>
__global__ void __launch_bounds__(256) cholesky_ragged_kernel(const CholTask* __restrict__ tasks) {
  const CholTask t = tasks[blockIdx.x];
  chol_one<C, 1>(t.N, t.A, t.mode, t.out, t.status, t.code, t.W, t.Vc, t.ldv);
}

// X = L^-1 for lower-triangular L (real positive diagonal), one CTA per
// (matrix, 32-column block): block forward substitution down the rows,
// X_r = L_rr^-1 (E_r - sum_{cb <= s < r} L_rs X_s); X is lower triangular.
template <bool C>
__global__ void __launch_bounds__(256) trinv_kernel(int N, const double* __restrict__ Lb, double* __restrict__ Xb) {
  __shared__ Elem<C> Ls[CB][CB + 1];
  __shared__ Elem<C> Xs[CB][CB + 1];
  const int nt = (N + CB - 1) / CB;
  const int b = blockIdx.x / nt, cb = blockIdx.x % nt;
  const long NN = (long)N * N;
  const double* L = Lb + (long)b * NN * (C ? 2 : 1);
  double* X = Xb + (long)b * NN * (C ? 2 : 1);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int c0 = cb * CB;
  const int ncol = min(CB, N - c0);
  for (long idx = tid; idx < (long)c0 * CB; idx += 256) {
    const int r = (int)(idx / CB), c = (int)(idx % CB);
    if (c < ncol) st_elem<C>(X, (long)r * N + c0 + c, zero_elem<C>());
  }
  for (int rb = cb; rb < nt; ++rb) {
    const int r0 = rb * CB;
    Elem<C> acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = zero_elem<C>();
    for (int sb = cb; sb < rb; ++sb) {
      const int s0 = sb * CB;
      for (int idx = tid; idx < CB * CB; idx += 256) {
        const int r = idx / CB, c = idx % CB;
        Ls[r][c] = (r0 + r < N) ? ld_elem<C>(L, (long)(r0 + r) * N + s0 + c) : zero_elem<C>();
        Xs[r][c] = (c < ncol) ? ld_elem<C>(X, (long)(s0 + r) * N + c0 + c) : zero_elem<C>();
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < CB; ++k) {
        const Elem<C> xv = Xs[k][tx];
#pragma unroll
        for (int u = 0; u < 4; ++u) mac<C>(acc[u], Ls[ty + 8 * u][k], xv);
      }
      __syncthreads();
    }
    // right-hand side E_r - acc, and the diagonal block of L
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = ty + 8 * u;
      Elem<C> e = zero_elem<C>();
      e.re = (r0 + r == c0 + tx) ? 1.0 : 0.0;
      e.re -= acc[u].re;
      if constexpr (C) e.im = -acc[u].im;
      Xs[r][tx] = e;
    }
    for (int idx = tid; idx < CB * CB; idx += 256) {
      const int r = idx / CB, c = idx % CB;
      Ls[r][c] = (r0 + r < N && r0 + c < N && c <= r) ? ld_elem<C>(L, (long)(r0 + r) * N + r0 + c) : zero_elem<C>();
    }
    __syncthreads();
    if (tid < CB) {
      const int c = tid;
      const int nr = min(CB, N - r0);
      for (int r = 0; r < nr; ++r) {
        Elem<C> v = Xs[r][c];
        for (int k = 0; k < r; ++k) {
          Elem<C> prod = zero_elem<C>();
          mac<C>(prod, Ls[r][k], Xs[k][c]);
          v.re -= prod.re;
          if constexpr (C) v.im -= prod.im;
        }
        const double d = Ls[r][r].re;
        v.re /= d;
        if constexpr (C) v.im /= d;
        Xs[r][c] = v;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < CB * CB; idx += 256) {
      const int r = idx / CB, c = idx % CB;
      if (r0 + r < N && c < ncol) st_elem<C>(X, (long)(r0 + r) * N + c0 + c, Xs[r][c]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- energy -----

__global__ void energy_kernel(int n_q, int n_w, const double* __restrict__ parts, const double* __restrict__ w_q,
                              const double* __restrict__ zeta_w, double* __restrict__ eps, double* __restrict__ Ec) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // Neumaier-compensated sums in a fixed order: q inside, frequency outside.
  double E = 0.0, Ec_c = 0.0;
  for (int w = 0; w < n_w; ++w) {
    double e = 0.0, c = 0.0;
    for (int q = 0; q < n_q; ++q) {
      const double v = parts[2 * ((long)q * n_w + w)] + parts[2 * ((long)q * n_w + w) + 1];
      eps[(long)q * n_w + w] = v;
      const double x = w_q[q] * v;
      const double t = e + x;
      c += (fabs(e) >= fabs(x)) ? (e - t) + x : (x - t) + e;
      e = t;
    }
    const double x = zeta_w[w] * (e + c);
    const double t = E + x;
    Ec_c += (fabs(E) >= fabs(x)) ? (E - t) + x : (x - t) + E;
    E = t;
  }
  *Ec = (E + Ec_c) / (2.0 * M_PI);
}

}  // namespace

// ------------------------------------------------------------ launchers ----

cudaError_t launch_dtab(const BatchGeom& g, const double* eps_occ, const double* eps_virt, const int* kidx,
                        const int* kqidx, const double* omega, double zeta_k, double* dtab, cudaStream_t s) {
  const long total = (long)g.n_qb * g.n_k * g.n_w * g.n_ov;
  if (total == 0) return cudaSuccess;
  const long blocks = std::min<long>((total + 255) / 256, 152L * 16);
  dtab_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, eps_occ, eps_virt, kidx, kqidx, omega, zeta_k, dtab);
  return cudaGetLastError();
}

cudaError_t launch_chi0_fp64(const BatchGeom& g, const double* const* Cptrs, const double* dtab, double* chi,
                             cudaStream_t s) {
  return g.cplx ? chi0_dispatch<true>(g, Cptrs, dtab, chi, s) : chi0_dispatch<false>(g, Cptrs, dtab, chi, s);
}

cudaError_t launch_sandwich(int cplx, int N, int n_batch, int n_w, const double* chi, const double* L, double* T,
                            double* Y, cudaStream_t s) {
  if (n_batch == 0) return cudaSuccess;
  const int nt = (N + GT - 1) / GT;
  const int full = nt * nt, tri = nt * (nt + 1) / 2;
  if (cplx) {
    sandwich_kernel<true, 0><<<n_batch * full, 256, 0, s>>>(N, n_w, chi, L, T, nt, full);
    sandwich_kernel<true, 1><<<n_batch * tri, 256, 0, s>>>(N, n_w, T, L, Y, nt, tri);
  } else {
    sandwich_kernel<false, 0><<<n_batch * full, 256, 0, s>>>(N, n_w, chi, L, T, nt, full);
    sandwich_kernel<false, 1><<<n_batch * tri, 256, 0, s>>>(N, n_w, T, L, Y, nt, tri);
  }
  return cudaGetLastError();
}

// Teams of CL_BIG CTAs per matrix when the launch has too few matrices to
// fill the GPU with one CTA each and the matrices are large enough to share.
constexpr int CL_BIG = 8;

template <bool C, int CL>
cudaError_t launch_chol_t(int N, int b0, int n_mat, double* mats, long bstride, int mode, double* out, int* status,
                          int status_base, cudaStream_t s, const double* Wn, const double* Vc, const double* ldV,
                          int n_w) {
  if constexpr (CL == 1) {
    cholesky_kernel<C, 1><<<n_mat, 256, 0, s>>>(N, mats, bstride, mode, out, status, status_base, Wn, Vc, ldV, n_w,
                                                 b0);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_mat * CL));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cholesky_kernel<C, CL>, N, mats, bstride, mode, out, status, status_base, Wn, Vc,
                              ldV, n_w, b0);
  }
  return cudaGetLastError();
}

// Clusters of CL CTAs of cholesky_kernel<C, CL> the current device holds at
// once (cudaOccupancyMaxActiveClusters), queried once per device (under a
// lock); 0 if the query fails.
template <bool C, int CL>
int chol_max_clusters() {
  static std::mutex mu;
  static int cache[MAX_DEVICES];
  static bool have[MAX_DEVICES] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= MAX_DEVICES) dev = 0;
  if (!have[dev]) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(256);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int m = 0;
    if (cudaOccupancyMaxActiveClusters(&m, cholesky_kernel<C, CL>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      m = 0;
    }
    cache[dev] = m;
    have[dev] = true;
  }
  return cache[dev];
}

// A cluster per matrix: CL_BIG CTAs each when all the launch's clusters fit
// on the device at once, else clusters of 4 when those do (one wave instead of
// two: the serial diagonal and panel phases, not the trailing update, set a
// cluster's time).
template <bool C>
cudaError_t launch_chol_clusters(int N, int b0, int n_mat, double* mats, long bstride, int mode, double* out,
                                 int* status, int status_base, cudaStream_t s, const double* Wn, const double* Vc,
                                 const double* ldV, int n_w) {
  const int m8 = chol_max_clusters<C, CL_BIG>();
  if (m8 > 0 && n_mat > m8 && chol_max_clusters<C, 4>() >= n_mat)
    return launch_chol_t<C, 4>(N, b0, n_mat, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV, n_w);
  return launch_chol_t<C, CL_BIG>(N, b0, n_mat, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV, n_w);
}

// The launch split of launch_chol_c: 0 = one CTA per matrix, 1 = a cluster
// per matrix, 2 = one CTA per matrix except a short last wave on clusters.
int chol_split(int N, int n_mat) {
  const int P = num_sms_fp64(), W = P * CHOL_CTAS_PER_SM;  // W: matrices in one wave
  if (N >= 256 && n_mat * 2 < P) return 1;
  const int r = n_mat % W;
  if (N >= 256 && n_mat > W && r > 0 && r * 2 < W) return 2;
  return 0;
}

template <bool C>
cudaError_t launch_chol_c(int N, int n_mat, double* mats, long bstride, int mode, double* out, int* status,
                          int status_base, cudaStream_t s, const double* Wn, const double* Vc, const double* ldV,
                          int n_w) {
  const int W = num_sms_fp64() * CHOL_CTAS_PER_SM;
  const int split = chol_split(N, n_mat);
  // few large matrices: a cluster per matrix
  if (split == 1)
    return launch_chol_clusters<C>(N, 0, n_mat, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV, n_w);
  // one CTA per matrix; a short last wave (fewer than P/2 matrices) goes to
  // clusters instead, so that it does not run on a few SMs alone
  const int r = n_mat % W;
  if (split == 2) {
    cudaError_t e = launch_chol_t<C, 1>(N, 0, n_mat - r, mats, bstride, mode, out, status, status_base, s, Wn, Vc,
                                        ldV, n_w);
    if (e != cudaSuccess) return e;
    return launch_chol_clusters<C>(N, n_mat - r, r, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV,
                                   n_w);
  }
  return launch_chol_t<C, 1>(N, 0, n_mat, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV, n_w);
}

cudaError_t launch_cholesky(int cplx, int N, int n_mat, double* mats, long bstride, int mode, double* out,
                            int* status, int status_base, cudaStream_t s, const double* Wn, const double* Vc,
                            const double* ldV, int n_w) {
  if (n_mat == 0) return cudaSuccess;
  if (mode == 2 && (!Wn || !Vc || !ldV || n_w <= 0)) return cudaErrorInvalidValue;
  if (cplx) return launch_chol_c<true>(N, n_mat, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV, n_w);
  return launch_chol_c<false>(N, n_mat, mats, bstride, mode, out, status, status_base, s, Wn, Vc, ldV, n_w);
}

int cholesky_launches(int N, int n_mat) { return n_mat <= 0 ? 0 : (chol_split(N, n_mat) == 2 ? 2 : 1); }

cudaError_t launch_cholesky_ragged(int cplx, const CholTask* tasks, int n_tasks, cudaStream_t s) {
  if (n_tasks <= 0) return cudaSuccess;
  if (cplx)
    cholesky_ragged_kernel<true><<<n_tasks, 256, 0, s>>>(tasks);
  else
    cholesky_ragged_kernel<false><<<n_tasks, 256, 0, s>>>(tasks);
  return cudaGetLastError();
}

cudaError_t launch_vinv(int cplx, int N, int n_q, const double* L, double* X, double* Wn, cudaStream_t s) {
  if (n_q == 0) return cudaSuccess;
  const int nb = (N + CB - 1) / CB;
  const int nt = (N + GT - 1) / GT, tri = nt * (nt + 1) / 2;
  if (cplx) {
    trinv_kernel<true><<<n_q * nb, 256, 0, s>>>(N, L, X);
    sandwich_kernel<true, 1><<<n_q * tri, 256, 0, s>>>(N, 1, X, X, Wn, nt, tri);
  } else {
    trinv_kernel<false><<<n_q * nb, 256, 0, s>>>(N, L, X);
    sandwich_kernel<false, 1><<<n_q * tri, 256, 0, s>>>(N, 1, X, X, Wn, nt, tri);
  }
  return cudaGetLastError();
}

cudaError_t launch_energy_reduce(int n_q, int n_w, const double* parts, const double* w_q, const double* zeta_w,
                                 double* eps, double* Ec, cudaStream_t s) {
  energy_kernel<<<1, 32, 0, s>>>(n_q, n_w, parts, w_q, zeta_w, eps, Ec);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) copy16_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) dst[i] = src[i];
}

cudaError_t launch_copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s, uint64_t* n_launch) {
  if (bytes == 0) return cudaSuccess;
  if (bytes % 16 || (uintptr_t)dst % 16 || (uintptr_t)src % 16)
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
  const long n = (long)(bytes / 16);
  const unsigned blocks = (unsigned)std::min<long>((n + 255) / 256, (long)num_sms_fp64() * 8);
  copy16_kernel<<<blocks, 256, 0, s>>>((uint4*)dst, (const uint4*)src, n);
  if (n_launch) ++*n_launch;
  return cudaGetLastError();
}

}  // namespace rpa
