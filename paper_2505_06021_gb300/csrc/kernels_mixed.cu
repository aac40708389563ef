// Split-precision chi0 on the tcgen05 tensor cores of GB300 (sm_103a).
//
// chi0_PQ(q, w) = - sum_t conj(A_Pt) C_Qt with A = zeta_k |d_t(w)| C (the
// fit-basis response of Sec. 2.2; d_t < 0) is a dense Hermitian contraction
// over t = (k, i, a).  The frequency weight sits on the A side only, so the B
// operand (slices of C itself) is built once per q and reused by every
// frequency; only A is re-sliced per frequency.
//
// Digit slices.  Each FP64 value x of row P becomes the fixed-point integer
// F = round(x 2^(31 - e_P)), |F| <= 2^30, e_P one exponent per row and
// frequency, computed from the FP64 bit patterns with integer arithmetic only
// (GB300's FP64 pipe runs at 1/58 of FP32).  F = d0 2^24 + d1 2^16 + d2 2^8 +
// d3 with |d0| <= 64, |d_i| <= 128; the BF16 slices v_i = d_i 2^(-8i) are exact
// and x = 2^(e_P - 7) sum_i v_i.
//
// Real embedding.  A complex row is stored interleaved, X = (re_0, im_0, re_1,
// im_1, ...), and the B operand of a tile stacks X_Q over Y_Q = (im_0, -re_0,
// ...) of C, so that one MMA of N = 128 gives [X_P X_Q^T | X_P Y_Q^T] =
// [Re | Im] of sum_t conj(A_P) C_Q for 64 columns Q.
//
// Exactness.  Slice pairs (i, j) with i + j <= s - 1 (plus (1, 1) for s = 2)
// are grouped by level into four TMEM accumulators: levels 0, 1 and 2 hold
// integer-valued sums that stay below 2^24 for CHUNK t (exact FP32
// accumulation whatever the tensor core's rounding), level 3 (2^-24 below
// level 0) is plain FP32.  Every CHUNK t the eight epilogue warps drain the four groups
// and add them into float-float (hi, lo) register accumulators.
//
// The tensor-core kernel itself is in chi0_tc.cuh.  The K range of each tile
// is split over CTAs (split-K); a reduction kernel here adds the partials in
// a fixed order, applies the exponents and writes chi0 in FP64 (lower
// triangle + Hermitian mirror), so results are deterministic.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "chi0_tc.cuh"
#include "rpa_internal.h"

namespace rpa {
namespace {

// ------------------------------------------------------------ slicing -----
// Fixed-point inputs, built once per q (C) and once per frequency table (w):
//   c_fix = round(c 2^(30 - eC_P)), |c| < 2^eC_P for the whole row P, |c_fix| <= 2^30;
//   w = w_m 2^(ew - 31) with w_m in [2^30, 2^31), one 31-bit mantissa per (k, t, w).
// Their digit planes are written by slice_unit (slice.cuh).

// c_fix of one q: [Npad][Kr] int32, zero outside the data; eC per row.
// Rows along grid y, K along grid x (both grid-stride), so that no element
// needs a 64-bit division; consecutive threads read consecutive values of C.
__global__ void __launch_bounds__(256) cfix_kernel(int cplx, int N, int Npad, int n_ov, int n_k, int Ktot, int Kr,
                                                   const double* const* C, const int* eC, int* cfix) {
  for (int P = blockIdx.y; P < Npad; P += gridDim.y) {
    int* out = cfix + (long)P * Kr;
    const int eP = P < N ? eC[P] : 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Kr; k += gridDim.x * blockDim.x) {
      const int tglob = cplx ? (k >> 1) : k;
      int v = 0;
      if (P < N && tglob < Ktot) {
        const int j = tglob / n_ov, t = tglob - j * n_ov;
        const double c = cplx ? C[j][2 * ((long)P * n_ov + t) + (k & 1)] : C[j][(long)P * n_ov + t];
        const unsigned long long cb = (unsigned long long)__double_as_longlong(c);
        const int Ec = (int)((cb >> 52) & 0x7ff);
        if (Ec != 0) {
          // c = mant 2^(Ec - 1075); c_fix = c 2^(30 - eC) = mant >> (1045 - Ec + eC), a shift of
          // at least 23 since eC >= Ec - 1022
          const int sh = 1045 - Ec + eP;
          const unsigned long long mant = (cb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
          if (sh < 64) {
            const int m = (int)((mant + (1ull << (sh - 1))) >> sh);
            v = (cb >> 63) ? -m : m;
          }
        }
      }
      out[k] = v;
    }
  }
}

template <bool CPLX, bool WEIGHTED>
__global__ void __launch_bounds__(256, 2) slice_kernel(SliceArgs a) {
  const long total = (long)a.Npad * (a.Kr / 16);
  // consecutive threads take consecutive rows of one K-block: coalesced
  // stores into the blocked layout, shared weight loads
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x)
    slice_unit<CPLX, WEIGHTED>(a, idx);
}

// Row exponents.  eA[w][P] = max_t (Ec_t + Ew_t) - 2044 + 1 (biased fields),
// so |c w| < 2^(eA - 1) on row P; eC[P] = max_t Ec_t - 1022, so |c| < 2^eC.
// Phase 1: block (rows 8 bx .. 8 bx + 7, part kp) covers k-point j = kp / TP
// and its t8-chunks [tp n8 / TP, (tp + 1) n8 / TP), tp = kp mod TP; warp w
// takes row 8 bx + w, lane l the l-th chunk of each group of 32 chunks.  The
// 16-bit weight exponents of a group (all frequencies) are staged in shared
// memory once for the block's 8 rows.  Each warp writes its row's raw maxima
// (Ec_t + Ew_t + 1022 per frequency, Ec_t; 0 where no entry is nonzero) to
// part[kp][g][P] (g = n_w: the Ec maximum).  Phase 2 takes the maximum over
// the parts.
constexpr int MAX_W = 32;
constexpr int EROW_ROWS = 8;
__global__ void __launch_bounds__(256) erow_part_kernel(int cplx, int N, int Npad, int n_ov, int n_w, int TP,
                                                        const double* const* C, const int16_t* ew, int* part) {
  __shared__ uint4 ews[MAX_W][32];  // [frequency][chunk of the group]: 8 exponents each
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = blockIdx.x * EROW_ROWS + warp, kp = blockIdx.y;
  const int j = kp / TP, tp = kp - j * TP;
  const int n8 = (n_ov + 7) / 8;
  const int c0 = (int)((long)tp * n8 / TP), c1 = (int)((long)(tp + 1) * n8 / TP);
  const bool vec = (n_ov % 8 == 0);
  const int16_t* ewj = ew + (long)j * n_w * n_ov;
  const unsigned long long* row =
      P < N ? reinterpret_cast<const unsigned long long*>(C[j]) + (long)P * n_ov * (cplx ? 2 : 1) : nullptr;
  int m[MAX_W];
  int mc = 0;
#pragma unroll
  for (int g = 0; g < MAX_W; ++g) m[g] = 0;
  for (int g0 = c0; g0 < c1; g0 += 32) {
    // stage the group's exponents: n_w x 32 chunks of 8 values
    for (int u = threadIdx.x; u < n_w * 32; u += blockDim.x) {
      const int g = u >> 5, ch = g0 + (u & 31);
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (ch < c1) {
        const int16_t* src = ewj + (long)g * n_ov + (long)ch * 8;
        if (vec) {
          v = *reinterpret_cast<const uint4*>(src);
        } else {
          int16_t tmp[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) tmp[e] = (ch * 8 + e < n_ov) ? src[e] : (int16_t)0;
          memcpy(&v, tmp, 16);
        }
      }
      ews[g][u & 31] = v;
    }
    __syncthreads();
    const int t8 = g0 + lane;
    if (row && t8 < c1) {
      int ec[8];
      int emax = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t8 * 8 + u;
        ec[u] = -100000;
        if (t < n_ov) {
          int e;
          if (cplx) {
            const ulonglong2 x = reinterpret_cast<const ulonglong2*>(row)[t];
            e = max((int)((x.x >> 52) & 0x7ff), (int)((x.y >> 52) & 0x7ff));
          } else {
            e = (int)((row[t] >> 52) & 0x7ff);
          }
          if (e != 0) ec[u] = e;
          emax = max(emax, e);
        }
      }
      mc = max(mc, emax);
      if (emax != 0) {
#pragma unroll
        for (int g = 0; g < MAX_W; ++g) {
          if (g >= n_w) break;
          const uint4 v = ews[g][lane];
          int16_t ev[8];
          memcpy(ev, &v, 16);
#pragma unroll
          for (int u = 0; u < 8; ++u) m[g] = max(m[g], ec[u] + (int)ev[u] + 1022);
        }
      }
    }
    __syncthreads();
  }
  // row maxima: one warp reduction per value
#pragma unroll
  for (int g = 0; g < MAX_W; ++g) {
    if (g >= n_w) break;
    const int r = __reduce_max_sync(0xffffffffu, m[g]);
    if (lane == 0 && P < Npad) part[((long)kp * (n_w + 1) + g) * Npad + P] = r;
  }
  const int r = __reduce_max_sync(0xffffffffu, mc);
  if (lane == 0 && P < Npad) part[((long)kp * (n_w + 1) + n_w) * Npad + P] = r;
}

__global__ void __launch_bounds__(256) erow_final_kernel(int n_w, int Npad, int KP, const int* part, int* eA,
                                                         int* eC) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (n_w + 1) * Npad) return;
  const int g = idx / Npad, P = idx - g * Npad;
  int r = 0;
  for (int kp = 0; kp < KP; ++kp) r = max(r, part[((long)kp * (n_w + 1) + g) * Npad + P]);
  if (g < n_w)
    eA[(long)g * Npad + P] = r > 0 ? r - 2044 + 1 : -2000;
  else
    eC[P] = r ? r - 1022 : -2000;
}

// w = zeta_k |d| as a 31-bit mantissa and exponent: w = wm 2^(ew - 31),
// wm in [2^30, 2^31); wx packs wm | (uint32) ew << 32 for the slicing.
__global__ void __launch_bounds__(256) wtab_kernel(long n, const double* dtab, unsigned long long* wx, int16_t* ew) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(dtab[i]));
    const int E = (int)((b >> 52) & 0x7ff);
    unsigned long long m = (((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) + (1ull << 21)) >> 22;  // [2^30, 2^31]
    int e = E - 1022;
    if (m >> 31) {
      m >>= 1;
      ++e;
    }
    const int ee = E ? e : -2000;
    wx[i] = (E ? m : 0ull) | ((unsigned long long)(uint32_t)ee << 32);
    ew[i] = (int16_t)ee;
  }
}

// Sum of the split-K partials in a fixed order, exponents, Hermitian store.
// Blocks: (segment, frequency, tile), enumerated through block0 offsets.
struct RedSeg {
  int cplx, N, Npad, n_tiles, n_ksplit, w0, G, block0;
  const float* part;
  const int* erow;   // [n_w][Npad] exponents of the weighted rows (A)
  const int* erowC;  // [Npad] exponents eC of C (B digits use e = eC + 1)
  double* chi;       // [n_w][N][N] of this q
};
struct RedParams {
  int n_segs;
  RedSeg seg[MAX_SEGS];
};
static_assert(sizeof(RedParams) <= 32000, "kernel parameter block too large");

__global__ void __launch_bounds__(256) reduce_kernel(const __grid_constant__ RedParams rp) {
  int sg = 0;
  while (sg + 1 < rp.n_segs && rp.seg[sg + 1].block0 <= (int)blockIdx.x) ++sg;
  const RedSeg& a = rp.seg[sg];
  const int b = blockIdx.x - a.block0;
  const int tile = b % a.n_tiles;
  const int g = b / a.n_tiles;
  int I, J;
  tile_ij(a.cplx, tile, I, J);
  const long NN = (long)a.N * a.N;
  double* out = a.chi + (long)(a.w0 + g) * NN * (a.cplx ? 2 : 1);
  const int ncols = a.cplx ? 64 : 128;
  for (int idx = threadIdx.x; idx < 128 * ncols; idx += blockDim.x) {
    const int r = idx / ncols, c = idx % ncols;
    const int P = I * 128 + r, Q = J * ncols + c;
    if (P >= a.N || Q >= a.N || Q > P) continue;
    double re = 0.0, im = 0.0;
    for (int ks = 0; ks < a.n_ksplit; ++ks) {
      const long item = ((long)ks * a.G + g) * a.n_tiles + tile;
      const float* pp = a.part + item * 2 * 128 * 128 + (long)r * 128;
      re += (double)pp[c] + (double)pp[128 * 128 + c];
      if (a.cplx) im += (double)pp[64 + c] + (double)pp[128 * 128 + 64 + c];
    }
    const int e = a.erow[(long)(a.w0 + g) * a.Npad + P] + a.erowC[Q] + 1;  // B side: e = eC + 1
    const double sc = -ldexp(1.0, e - 14);  // x = 2^(e - 7) sum v, chi = -sum conj(a) c
    re *= sc;
    im *= sc;
    if (a.cplx) {
      if (P == Q) im = 0.0;
      reinterpret_cast<double2*>(out)[(long)P * a.N + Q] = make_double2(re, im);
      if (P != Q) reinterpret_cast<double2*>(out)[(long)Q * a.N + P] = make_double2(re, -im);
    } else {
      out[(long)P * a.N + Q] = re;
      if (P != Q) out[(long)Q * a.N + P] = re;
    }
  }
}

// A time-out inside the tensor-core kernel becomes a status word code.
__global__ void err_merge_kernel(const int* err, int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *err != 0) atomicCAS(status, 0, 1 + (1 << 30) + *err);
}

// ------------------------------------------------------------ host side --

int num_sms() { return device_sm_count(); }

// Workspace of one q: slices of A for up to G frequencies, slices of C,
// exponents, fixed-point C, weights, split-K partials.
struct MixedLayout {
  int Npad, Ktot, Kr, nxy, G, n_tiles, n_kb, n_chunks, nks_cap, TP, KP;
  size_t slices, slicesC, erow, erowC, part, wm, ew, cfix, erowp, total;
};

constexpr int KB_PER_CHUNK = 2 * CHUNK / KB;

// slice_cap: bytes allowed for the A slices of one q (bounds G, the number of
// frequencies per launch).  The partial buffer is sized for the largest split
// count any launch of this q may use (nks_cap).
MixedLayout mixed_layout(const BatchGeom& g, int s, int sms, size_t slice_cap) {
  MixedLayout L{};
  L.Npad = (g.n_aux + 127) / 128 * 128;
  L.Ktot = g.n_k * g.n_ov;
  const int chunk_t = g.cplx ? CHUNK : 2 * CHUNK;  // t per exact chunk (2048 real values)
  const int Kt = (L.Ktot + chunk_t - 1) / chunk_t * chunk_t;
  L.Kr = g.cplx ? 2 * Kt : Kt;  // real K (interleaved re, im)
  L.nxy = g.cplx ? 2 : 1;
  L.n_kb = L.Kr / KB;
  L.n_chunks = L.n_kb / KB_PER_CHUNK;
  const int nb = L.Npad / 128;
  L.n_tiles = g.cplx ? nb * (nb + 1) : nb * (nb + 1) / 2;
  const size_t per_w = (size_t)s * L.Npad * L.Kr * 2;  // A: X planes only
  const size_t gmax = std::max<size_t>(1, slice_cap / per_w);
  L.G = (int)std::min<size_t>((size_t)std::min(g.n_w, MAX_W), gmax);
  L.nks_cap = std::max(1, std::min(L.n_chunks, (8 * sms + L.G * L.n_tiles - 1) / (L.G * L.n_tiles)));
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  L.slices = al(per_w * L.G);
  L.slicesC = al(per_w * L.nxy);
  L.erow = al(sizeof(int) * (size_t)g.n_w * L.Npad);
  L.erowC = al(sizeof(int) * (size_t)L.Npad);
  L.part = al(sizeof(float) * 2 * 128 * 128 * (size_t)L.G * L.n_tiles * L.nks_cap);
  L.wm = al(sizeof(unsigned long long) * (size_t)g.n_k * g.n_w * g.n_ov);
  L.ew = al(sizeof(int16_t) * (size_t)g.n_k * g.n_w * g.n_ov);
  L.cfix = al(sizeof(int) * (size_t)L.Npad * L.Kr);
  // row-exponent parts: at least 8 per row (a k-point's t range is cut in TP pieces)
  L.TP = g.n_k >= 8 ? 1 : (8 + g.n_k - 1) / g.n_k;
  L.KP = g.n_k * L.TP;
  L.erowp = al(sizeof(int) * (size_t)L.KP * (g.n_w + 1) * L.Npad);
  L.total = L.slices + L.slicesC + L.erow + L.erowC + L.part + L.wm + L.ew + L.cfix + L.erowp;
  return L;
}

// Accumulator groups used by s slices: levels 0 .. s-1, plus level 2 for the
// (1, 1) pair of s = 2, capped at the last group (MmaTable's rule).
constexpr int group_mask(int s) {
  int m = 0;
  for (int lvl = 0; lvl < s; ++lvl) m |= 1 << (lvl < NGROUPS - 1 ? lvl : NGROUPS - 1);
  if (s == 2) m |= 1 << 2;
  return m;
}
static_assert(group_mask(2) == MmaTable<2>{}.mask && group_mask(3) == MmaTable<3>{}.mask &&
                  group_mask(4) == MmaTable<4>{}.mask,
              "host and kernel accumulator groups disagree");

// ---------------------------------------------------- split-K planning ----
// A launch's segments get their split-K depth from one common target item
// length Lc (in exact 2048-value chunks): a segment of n chunks is cut into
// nks = ceil(n / Lc) splits (at most nks_cap), so long and short segments give
// items of similar length.  Items are issued to CTAs round robin, longest
// segments first; the model cost of a plan is the largest per-CTA sum of item
// lengths plus a fixed per-item overhead (pipeline fill, partial store).

struct SegShape {
  int n_chunks, G, T, nks_cap;
};

struct SplitPlan {
  std::vector<int> nks;  // per segment
  std::vector<int> order;
  double cost;
};

SplitPlan plan_for(const std::vector<SegShape>& v, int Lc, int sms) {
  SplitPlan p;
  const int n = (int)v.size();
  p.nks.resize(n);
  std::vector<int> cps(n);
  long items = 0;
  for (int i = 0; i < n; ++i) {
    int k = std::min(v[i].nks_cap, std::max(1, (v[i].n_chunks + Lc - 1) / Lc));
    cps[i] = (v[i].n_chunks + k - 1) / k;
    k = (v[i].n_chunks + cps[i] - 1) / cps[i];
    p.nks[i] = k;
    items += (long)k * v[i].G * v[i].T;
  }
  p.order.resize(n);
  for (int i = 0; i < n; ++i) p.order[i] = i;
  std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) { return cps[a] > cps[b]; });
  const int grid = (int)std::max<long>(1, std::min<long>(items, sms));
  std::vector<double> load(grid, 0.0);
  long it = 0;
  for (int oi = 0; oi < n; ++oi) {
    const int i = p.order[oi];
    for (int ks = 0; ks < p.nks[i]; ++ks) {
      const int len = std::min(cps[i], v[i].n_chunks - ks * cps[i]);
      const long cnt = (long)v[i].G * v[i].T;
      // cnt consecutive items of equal length: whole rounds over the grid
      // plus a remainder starting at CTA it % grid
      const long full = cnt / grid, rem = cnt % grid;
      const double w = len + 0.3;
      if (full)
        for (int b = 0; b < grid; ++b) load[b] += full * w;
      for (long r = 0; r < rem; ++r) load[(it + r) % grid] += w;
      it += cnt;
    }
  }
  p.cost = *std::max_element(load.begin(), load.end());
  return p;
}

// Candidate target lengths: the values of Lc at which some segment's split
// count changes.
std::vector<int> candidates(const std::vector<SegShape>& v) {
  std::vector<int> c;
  for (const SegShape& s : v)
    for (int k = 1; k <= s.nks_cap; ++k) c.push_back((s.n_chunks + k - 1) / k);
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  if (c.size() > 48) {  // thin out evenly, keeping both ends
    std::vector<int> d;
    for (int i = 0; i < 48; ++i) d.push_back(c[(size_t)i * (c.size() - 1) / 47]);
    d.erase(std::unique(d.begin(), d.end()), d.end());
    c.swap(d);
  }
  return c;
}

uint64_t round_key(const std::vector<SegShape>& v, int s) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)s;
  auto mix = [&](uint64_t x) {
    h ^= x;
    h *= 1099511628211ull;
  };
  for (const SegShape& q : v) {
    mix((uint64_t)q.n_chunks);
    mix((uint64_t)q.G);
    mix((uint64_t)q.T);
    mix((uint64_t)q.nks_cap);
  }
  return h;
}

void launch_slice(int cplx, unsigned grid, cudaStream_t st, const SliceArgs& a) {
  if (a.wx) {
    if (cplx)
      slice_kernel<true, true><<<grid, 256, 0, st>>>(a);
    else
      slice_kernel<false, true><<<grid, 256, 0, st>>>(a);
  } else {
    if (cplx)
      slice_kernel<true, false><<<grid, 256, 0, st>>>(a);
    else
      slice_kernel<false, false><<<grid, 256, 0, st>>>(a);
  }
}

// Tensor-core flops issued by every chi0_tc_kernel launch of this process
// (slice pairs x padded tiles x padded K of each segment).
std::atomic<unsigned long long> g_tc_flops{0};

void launch_tc(int s, int grid, size_t smem, cudaStream_t st, const TcParams& tp) {
  const unsigned long long pairs = (unsigned long long)(s * (s + 1) / 2 + (s == 2 ? 1 : 0));
  unsigned long long f = 0;
  for (int i = 0; i < tp.n_segs; ++i)
    f += (unsigned long long)tp.seg[i].G * tp.seg[i].n_tiles * (unsigned long long)tp.seg[i].n_kb * pairs * 2ull *
         128ull * 128ull * (unsigned long long)KB;
  g_tc_flops += f;
  if (s == 2)
    chi0_tc_kernel<2><<<grid, THREADS, smem, st>>>(tp);
  else if (s == 3)
    chi0_tc_kernel<3><<<grid, THREADS, smem, st>>>(tp);
  else
    chi0_tc_kernel<4><<<grid, THREADS, smem, st>>>(tp);
}

size_t slice_cap_of(const MixedQ& q) { return q.slice_cap ? q.slice_cap : ((size_t)12 << 30); }

constexpr size_t TC_SMEM = STAGES * STAGE_BYTES + 1024 + 256;  // stages, alignment pad, barriers

cudaError_t tc_smem_attr() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(chi0_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(chi0_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(chi0_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  });
  return attr;
}

// One q's workspace region (layout L) carved from p.
struct QState {
  MixedLayout L;
  uint16_t *S, *SC;
  int *erow, *erowC, *cfix, *erowp;
  unsigned long long* wx;
  int16_t* ew;
  float* part;
  int w_next, rounds_left;
};

QState carve_q(char* p, const MixedLayout& L, int n_w) {
  QState q;
  q.L = L;
  q.S = (uint16_t*)p;
  p += L.slices;
  q.SC = (uint16_t*)p;
  p += L.slicesC;
  q.erow = (int*)p;
  p += L.erow;
  q.erowC = (int*)p;
  p += L.erowC;
  q.part = (float*)p;
  p += L.part;
  q.wx = (unsigned long long*)p;
  p += L.wm;
  q.ew = (int16_t*)p;
  p += L.ew;
  q.cfix = (int*)p;
  p += L.cfix;
  q.erowp = (int*)p;
  q.w_next = 0;
  q.rounds_left = (n_w + L.G - 1) / L.G;
  return q;
}

constexpr int PREP_LAUNCHES = 5;

unsigned slice_grid(const MixedLayout& L, int sms) {
  const long tg = (long)L.Npad * (L.Kr / 16);
  return (unsigned)std::min<long>((tg + 255) / 256, (long)sms * 32);
}

// Per-q preparation (PREP_LAUNCHES launches): packed weights, row exponents
// (two phases), fixed-point C and the digit planes of C (the B operand).
void prep_q(const QState& q, const MixedQ& m, int s, int sms, cudaStream_t st) {
  const BatchGeom& g = m.g;
  const long nwt = (long)g.n_k * g.n_w * g.n_ov;
  wtab_kernel<<<(unsigned)std::min<long>((nwt + 255) / 256, (long)sms * 16), 256, 0, st>>>(nwt, m.dtab, q.wx, q.ew);
  erow_part_kernel<<<dim3((unsigned)((q.L.Npad + EROW_ROWS - 1) / EROW_ROWS), (unsigned)q.L.KP), 256, 0, st>>>(
      g.cplx, g.n_aux, q.L.Npad, g.n_ov, g.n_w, q.L.TP, m.Cptrs, q.ew, q.erowp);
  erow_final_kernel<<<((g.n_w + 1) * q.L.Npad + 255) / 256, 256, 0, st>>>(g.n_w, q.L.Npad, q.L.KP, q.erowp, q.erow,
                                                                           q.erowC);
  const int gy = std::min(q.L.Npad, 65535);
  const int gx = std::max(1, std::min((q.L.Kr + 255) / 256, sms * 32 / gy));
  cfix_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(g.cplx, g.n_aux, q.L.Npad, g.n_ov, g.n_k,
                                                                   q.L.Ktot, q.L.Kr, m.Cptrs, q.erowC, q.cfix);
  SliceArgs sc{g.cplx, q.L.Npad, g.n_ov, q.L.Ktot, q.L.Kr, s, g.n_w, 0, 1, q.L.nxy, q.cfix, q.erowC,
               nullptr, q.erow, q.SC};
  launch_slice(g.cplx, slice_grid(q.L, sms), st, sc);
}

// Weighted digit planes of frequencies [w0, w0 + G) of q into q.S.
SliceArgs weighted_args(const QState& q, const MixedQ& m, int s, int w0, int G) {
  const BatchGeom& g = m.g;
  return SliceArgs{g.cplx, q.L.Npad, g.n_ov, q.L.Ktot, q.L.Kr, s, g.n_w, w0, G, 1, q.cfix, q.erowC,
                   q.wx, q.erow, q.S};
}

}  // namespace

bool mixed_supported() { return true; }

uint64_t mixed_tensor_flops_issued() { return g_tc_flops.load(); }

// Test hook (rpa_test_drop_copy): the next tensor-core launch in this process
// leaves the first K-block of one work item unloaded.
static std::atomic<int> g_drop_item{-1};
void mixed_test_drop_arm(int item) { g_drop_item.store(item); }
int mixed_test_drop_take() { return g_drop_item.exchange(-1); }

size_t mixed_workspace_bytes(const BatchGeom& g, int n_slices, size_t slice_cap) {
  return 1024 + mixed_layout(g, n_slices, num_sms(), slice_cap).total;
}

uint64_t mixed_tensor_flops(const BatchGeom& g, int s) {
  const MixedLayout L = mixed_layout(g, s, num_sms(), (size_t)12 << 30);
  const int np = s * (s + 1) / 2 + (s == 2 ? 1 : 0);
  return (uint64_t)g.n_w * L.n_tiles * (uint64_t)L.n_kb * np * 2ull * 128 * 128 * KB;
}

size_t mixed_multi_workspace_bytes(const MixedQ* qs, int n, int s) {
  size_t t = 1024;
  for (int i = 0; i < n; ++i) t += mixed_layout(qs[i].g, s, num_sms(), slice_cap_of(qs[i])).total;
  return t;
}

// Several q (of one job or of many) share each persistent tensor-core launch.
// Per-q preparation runs first (weights, exponents, fixed-point C, digits of
// C); then, in rounds, every q that still has frequencies left writes the
// digits of its next frequency group and contributes one segment; one
// chi0_tc_kernel covers all segments of the round and one reduce_kernel
// finishes them.  Each q has its own workspace region.  With tune set (never
// under stream capture), the first round of each new shape class times the
// best few split plans and records the fastest.
cudaError_t launch_chi0_mixed_multi(const MixedQ* qs, int n, int s, void* work, size_t work_bytes, int* status,
                                    uint64_t* n_launch, cudaStream_t st, bool tune, const LaunchHook* hook) {
  auto hb = [&]() {
    if (hook) hook->begin(hook->user, st);
  };
  auto he = [&](int cls, int nk) {
    if (hook) hook->end(hook->user, st, cls, nk);
  };
  if (n <= 0) return cudaSuccess;
  if (s < 2 || s > MAX_S) return cudaErrorInvalidValue;
  const int sms = num_sms();
  const size_t smem = TC_SMEM;
  if (cudaError_t ea = tc_smem_attr()) return ea;
  std::vector<QState> Q(n);
  char* p = (char*)work;
  int* err = (int*)p;
  p += 1024;
  size_t used = 1024;
  for (int i = 0; i < n; ++i) {
    const BatchGeom& g = qs[i].g;
    if (g.n_w > MAX_W || g.n_w <= 0) return cudaErrorInvalidValue;
    const MixedLayout L = mixed_layout(g, s, sms, slice_cap_of(qs[i]));
    used += L.total;
    if (used > work_bytes) return cudaErrorMemoryAllocation;
    Q[i] = carve_q(p, L, g.n_w);
    p += L.total;
  }
  uint64_t nl = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return e;
  hb();
  for (int i = 0; i < n; ++i) {
    prep_q(Q[i], qs[i], s, sms, st);
    nl += PREP_LAUNCHES;
  }
  he(RPA_K_SLICE, PREP_LAUNCHES * n);
  TcParams tp;
  RedParams rp;
  while (true) {
    // this round's segments: every q with frequencies left, its next group
    // (groups spread evenly over the q's rounds)
    std::vector<int> who;
    std::vector<int> w0s, Gs;
    std::vector<SegShape> shp;
    for (int i = 0; i < n && (int)who.size() < MAX_SEGS; ++i) {
      QState& q = Q[i];
      const BatchGeom& g = qs[i].g;
      if (q.w_next >= g.n_w) continue;
      const int left = g.n_w - q.w_next;
      const int G = (left + q.rounds_left - 1) / q.rounds_left;
      who.push_back(i);
      w0s.push_back(q.w_next);
      Gs.push_back(G);
      shp.push_back(SegShape{q.L.n_chunks, G, q.L.n_tiles, q.L.nks_cap});
      q.w_next += G;
      q.rounds_left -= 1;
    }
    if (who.empty()) break;
    hb();
    for (size_t k = 0; k < who.size(); ++k) {
      const int i = who[k];
      launch_slice(qs[i].g.cplx, slice_grid(Q[i].L, sms), st, weighted_args(Q[i], qs[i], s, w0s[k], Gs[k]));
      ++nl;
    }
    he(RPA_K_SLICE, (int)who.size());
    // split plan: tuned value for this shape class if recorded, else the model's best
    const uint64_t key = round_key(shp, s);
    const std::vector<int> cand = candidates(shp);
    std::vector<std::pair<double, int>> ranked;
    for (int Lc : cand) ranked.push_back({plan_for(shp, Lc, sms).cost, Lc});
    std::stable_sort(ranked.begin(), ranked.end());
    int Lc = autotune_lookup(key);
    const bool do_tune = tune && Lc <= 0 && ranked.size() > 1;
    if (Lc <= 0) Lc = ranked[0].second;
    // builds both parameter blocks for target length Lc; returns the item count
    auto build = [&](int Lc_, int& items, int& blocks) -> bool {
      const SplitPlan pl = plan_for(shp, Lc_, sms);
      memset(&tp, 0, sizeof tp);
      memset(&rp, 0, sizeof rp);
      tp.s = s;
      tp.kb_per_chunk = KB_PER_CHUNK;
      tp.drop_item = mixed_test_drop_take();
      tp.err = err;
      tp.grp_mask = group_mask(s);
      items = 0;
      blocks = 0;
      for (int oi = 0; oi < (int)who.size(); ++oi) {
        const int k = pl.order[oi];
        const int i = who[k];
        QState& q = Q[i];
        const BatchGeom& g = qs[i].g;
        const int nks = pl.nks[k];
        const int cps = (q.L.n_chunks + nks - 1) / nks;
        TcSeg& S = tp.seg[tp.n_segs++];
        S.A = q.S;
        S.B = q.SC;
        S.nI = q.L.Npad / 128;
        S.part = q.part;
        S.cplx = g.cplx;
        S.G = Gs[k];
        S.n_tiles = q.L.n_tiles;
        S.n_ksplit = nks;
        S.kb_per_split = cps * KB_PER_CHUNK;
        S.n_kb = q.L.n_kb;
        S.kb_off = 0;
        S.ldb = q.L.n_kb;
        S.item0 = items;
        items += Gs[k] * q.L.n_tiles * nks;
        rp.seg[rp.n_segs++] = RedSeg{g.cplx, g.n_aux, q.L.Npad, q.L.n_tiles, nks, w0s[k], Gs[k], blocks,
                                     q.part, q.erow, q.erowC, qs[i].chi};
        blocks += Gs[k] * q.L.n_tiles;
      }
      tp.n_items = items;
      rp.n_segs = tp.n_segs;
      return true;
    };
    int items = 0, blocks = 0;
    if (do_tune) {
      cudaEvent_t e0, e1;
      if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
      if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
      float best = 1e30f;
      int bestLc = Lc;
      const size_t ntry = std::min<size_t>(4, ranked.size());
      for (size_t c = 0; c < ntry && e == cudaSuccess; ++c) {
        if (!build(ranked[c].second, items, blocks)) return cudaErrorInvalidValue;
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {  // first run warms L2 and the instruction cache
          cudaEventRecord(e0, st);
          launch_tc(s, std::min(items, sms), smem, st, tp);
          cudaEventRecord(e1, st);
          nl += 1;
          if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          ms = std::min(ms, t);
        }
        if (ms < best) {
          best = ms;
          bestLc = ranked[c].second;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (e != cudaSuccess) return e;
      Lc = bestLc;
      autotune_record(key, Lc);
    }
    if (!build(Lc, items, blocks)) return cudaErrorInvalidValue;
    hb();
    launch_tc(s, std::min(items, sms), smem, st, tp);
    he(RPA_K_CHI0, 1);
    hb();
    reduce_kernel<<<blocks, 256, 0, st>>>(rp);
    he(RPA_K_CHI0_RED, 1);
    nl += 2;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (status) {
    err_merge_kernel<<<1, 32, 0, st>>>(err, status);
    ++nl;
  }
  if (n_launch) *n_launch = nl;
  return cudaSuccess;
}

size_t mixed_seq_workspace_bytes(const BatchGeom& g, int n_slices, size_t slice_cap) {
  const MixedLayout L = mixed_layout(g, n_slices, num_sms(), slice_cap);
  if (L.G < g.n_w) return 1024 + L.total;  // several rounds per q: one region
  return 1024 + 2 * L.total;
}

// chi0 of n q of one geometry, one q after another, each in a single round
// (all its frequencies).  Two workspace regions alternate; the slicer warps
// of q's tensor-core launch write the weighted digit planes of the next q
// into the other region while q's MMAs run, so only the first q's weighted
// slicing is a launch of its own.  The next q's preparation (weights,
// exponents, fixed-point C, digits of C) runs before q's launch.  Falls back
// to one launch_chi0_mixed_multi call per q when the workspace cannot hold two
// single-round regions, the q differ in shape, or a launch would not fill the
// GPU (the two slicer warps of each CTA must share the slicing with every SM).
cudaError_t launch_chi0_mixed_seq(const MixedQ* qs, int n, int s, void* work, size_t work_bytes, int* status,
                                  uint64_t* n_launch, cudaStream_t st, const LaunchHook* hook) {
  auto hb = [&]() {
    if (hook) hook->begin(hook->user, st);
  };
  auto he = [&](int cls, int nk) {
    if (hook) hook->end(hook->user, st, cls, nk);
  };
  if (n <= 0) return cudaSuccess;
  if (s < 2 || s > MAX_S) return cudaErrorInvalidValue;
  const int sms = num_sms();
  const BatchGeom& g = qs[0].g;
  const size_t cap = slice_cap_of(qs[0]);
  const MixedLayout L = mixed_layout(g, s, sms, cap);
  const std::vector<SegShape> shp{SegShape{L.n_chunks, g.n_w, L.n_tiles, L.nks_cap}};
  int Lc = autotune_lookup(round_key(shp, s));
  if (Lc <= 0) {
    double best = 1e300;
    for (int c : candidates(shp)) {
      const double cost = plan_for(shp, c, sms).cost;
      if (cost < best) {
        best = cost;
        Lc = c;
      }
    }
  }
  const SplitPlan pl = plan_for(shp, Lc, sms);
  const int nks = pl.nks[0];
  const int n_items = g.n_w * L.n_tiles * nks;
  bool seq = n >= 2 && g.n_w > 0 && g.n_w <= MAX_W && L.G >= g.n_w && 1024 + 2 * L.total <= work_bytes &&
             n_items >= sms;
  for (int i = 1; i < n && seq; ++i) {
    const BatchGeom& h = qs[i].g;
    seq = h.cplx == g.cplx && h.n_aux == g.n_aux && h.n_occ == g.n_occ && h.n_virt == g.n_virt &&
          h.n_ov == g.n_ov && h.n_k == g.n_k && h.n_w == g.n_w && slice_cap_of(qs[i]) == cap;
  }
  if (!seq) {
    uint64_t tot = 0;
    for (int i = 0; i < n; ++i) {
      uint64_t nl = 0;
      const cudaError_t e = launch_chi0_mixed_multi(&qs[i], 1, s, work, work_bytes, status, &nl, st, false, hook);
      tot += nl;
      if (e != cudaSuccess) {
        if (n_launch) *n_launch = tot;
        return e;
      }
    }
    if (n_launch) *n_launch = tot;
    return cudaSuccess;
  }
  if (cudaError_t ea = tc_smem_attr()) return ea;
  char* p = (char*)work;
  int* err = (int*)p;
  QState R[2] = {carve_q(p + 1024, L, g.n_w), carve_q(p + 1024 + L.total, L, g.n_w)};
  uint64_t nl = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return e;
  hb();
  prep_q(R[0], qs[0], s, sms, st);
  launch_slice(g.cplx, slice_grid(L, sms), st, weighted_args(R[0], qs[0], s, 0, g.n_w));
  he(RPA_K_SLICE, PREP_LAUNCHES + 1);
  nl += PREP_LAUNCHES + 1;
  const int cps = (L.n_chunks + nks - 1) / nks;
  for (int i = 0; i < n; ++i) {
    const QState& c = R[i & 1];
    const bool more = i + 1 < n;
    if (more) {
      hb();
      prep_q(R[(i + 1) & 1], qs[i + 1], s, sms, st);
      he(RPA_K_SLICE, PREP_LAUNCHES);
      nl += PREP_LAUNCHES;
    }
    TcParams tp;
    RedParams rp;
    memset(&tp, 0, sizeof tp);
    memset(&rp, 0, sizeof rp);
    tp.s = s;
    tp.kb_per_chunk = KB_PER_CHUNK;
    tp.drop_item = mixed_test_drop_take();
    tp.err = err;
    tp.grp_mask = group_mask(s);
    tp.n_segs = 1;
    TcSeg& S = tp.seg[0];
    S.A = c.S;
    S.B = c.SC;
    S.nI = L.Npad / 128;
    S.part = c.part;
    S.cplx = g.cplx;
    S.G = g.n_w;
    S.n_tiles = L.n_tiles;
    S.n_ksplit = nks;
    S.kb_per_split = cps * KB_PER_CHUNK;
    S.n_kb = L.n_kb;
    S.kb_off = 0;
    S.ldb = L.n_kb;
    S.item0 = 0;
    tp.n_items = n_items;
    tp.side_on = more ? 1 : 0;
    if (more) tp.side = weighted_args(R[(i + 1) & 1], qs[i + 1], s, 0, g.n_w);
    rp.n_segs = 1;
    rp.seg[0] = RedSeg{g.cplx, g.n_aux, L.Npad, L.n_tiles, nks, 0, g.n_w, 0, c.part, c.erow, c.erowC, qs[i].chi};
    hb();
    launch_tc(s, std::min(n_items, sms), TC_SMEM, st, tp);
    he(RPA_K_CHI0, 1);
    hb();
    reduce_kernel<<<g.n_w * L.n_tiles, 256, 0, st>>>(rp);
    he(RPA_K_CHI0_RED, 1);
    nl += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (status) {
    err_merge_kernel<<<1, 32, 0, st>>>(err, status);
    ++nl;
  }
  if (n_launch) *n_launch = nl;
  return cudaSuccess;
}

cudaError_t launch_chi0_mixed(const BatchGeom& g, int s, const double* const* Cptrs, const double* dtab,
                              double* chi, void* work, size_t work_bytes, int* status, uint64_t* n_launch,
                              cudaStream_t st, size_t slice_cap, const LaunchHook* hook) {
  MixedQ q{g, Cptrs, dtab, chi, slice_cap};
  return launch_chi0_mixed_multi(&q, 1, s, work, work_bytes, status, n_launch, st, false, hook);
}

}  // namespace rpa

#include "chi0_binned.cuh"
