// Frequency-batched split-precision chi0 (device side and launcher).
//
// For one q the plan (freq_plan.cu) splits the transitions t = (k-pair, i, a)
// into bins of their energy D_t and gives each bin b a few skeleton
// frequencies; chi0(w) = sum_b sum_r coef[b][r][w] X_{b,r} with X_{b,r} the
// weighted contraction of bin b's transitions at skeleton r.  On the device:
//   1. ecrow_kernel     row maxima of C's exponent field (natural order);
//   2. perm_kernel      every transition's position in bin order (a warp per
//                       (k-pair, i) row, ranks by warp matching, stable) and
//                       its energy at that position;
//   3. wskel_kernel     the skeleton weights zeta_k |d(D_u, w_skel)| per
//                       position, packed as 31-bit mantissa and exponent;
//   4. cfix_scatter_kernel  fixed-point C, read in its natural order
//                       (coalesced) and written to the bin-order positions;
//   5. erow_bin_kernel  the row maxima of the weighted operand per (bin,
//                       skeleton), from the fixed-point values in bin order;
//   6. slice_kernel     the digit planes of C (the B operand, unchanged code);
//   7. per round: slice_bin_kernel (bin b's weighted planes for its skeletons
//      of the round) and one chi0_tc_kernel whose segments are the bins (each
//      reads B at its own K offset);
//   8. reduce_bin_kernel: per element the split-K partials of every (b, r),
//      scaled by their exponents and combined with coef into all n_w
//      frequencies in FP64, Hermitian store.
// With all skeletons in one round and two workspace regions, q+1's weighted
// planes are written by the slicer warps of q's tensor-core launch (its
// steps 1-6 run before that launch).  Included by kernels_mixed.cu.
#pragma once

namespace rpa {
namespace {

static_assert(SB_MAX_BINS == FREQ_MAX_BINS, "bin limits of the slicer and the plan differ");
constexpr int BIN_MAX_RANK = 32;  // skeletons per bin at most (= the frequency limit)
constexpr int STATUS_PLAN = STATUS_CODE_PLAN;  // device bin counts disagree with the plan

struct BinEdges {
  double edge[SB_MAX_BINS];
};

// Row maxima of the FP64 exponent field of C over all k-pairs of the q.
// Block: 8 rows (a warp each) x one part of one k-pair's row.
__global__ void __launch_bounds__(256) ecrow_kernel(int cplx, int N, int n_ov, int TP, const double* const* C,
                                                    int* eCraw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = blockIdx.x * 8 + warp;
  if (P >= N) return;
  const int j = blockIdx.y / TP, tp = blockIdx.y - j * TP;
  const long nv = (long)n_ov * (cplx ? 2 : 1);
  const long v0 = tp * nv / TP, v1 = (tp + 1) * nv / TP;
  const unsigned long long* row = reinterpret_cast<const unsigned long long*>(C[j]) + (long)P * nv;
  int m = 0;
  for (long v = v0 + lane; v < v1; v += 32) m = max(m, (int)((row[v] >> 52) & 0x7ff));
  m = __reduce_max_sync(0xffffffffu, m);
  if (lane == 0 && m > 0) atomicMax(eCraw + P, m);
}

// Position of every transition in bin order.  One warp per (k-pair jj,
// occupied i) row; bin b's transitions of the row go, in order of a, to
// rowoff[row][b] .. rowoff[row][b] + cnt[row][b] - 1 (both from the host
// plan): inv[jj n_ov + t] = position (-1 if not placed), dpos[position] = D
// (dpos stays 0 at padding positions).  A count that disagrees with the plan
// sets the status word and the position is not written (no access outside
// the bin's range).
__global__ void __launch_bounds__(256) perm_kernel(int n_k, int n_occ, int n_virt, int nb,
                                                   const __grid_constant__ BinEdges e, const double* eps_occ,
                                                   const double* eps_virt, const int* kidx, const int* kqidx,
                                                   const int* rowtab, int* inv, double* dpos, int* status) {
  __shared__ int run[8][SB_MAX_BINS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long nrow = (long)n_k * n_occ;
  const long row = (long)blockIdx.x * 8 + warp;
  if (row >= nrow) return;
  const int jj = (int)(row / n_occ), i = (int)(row - (long)jj * n_occ);
  if (lane < SB_MAX_BINS) run[warp][lane] = 0;
  __syncwarp();
  const double eo = eps_occ[(long)kidx[jj] * n_occ + i];
  const double* ev = eps_virt + (long)kqidx[jj] * n_virt;
  const int* off = rowtab + row * nb;
  const int* cnt = rowtab + (nrow + row) * nb;
  const int n_ov = n_occ * n_virt;
  for (int a0 = 0; a0 < n_virt; a0 += 32) {
    const int a = a0 + lane;
    const bool act = a < n_virt;
    double D = 0.0;
    int b = -1;
    if (act) {
      D = ev[a] - eo;
      b = 0;
      while (b < nb - 1 && D >= e.edge[b]) ++b;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int below = __popc(peers & ((1u << lane) - 1u));
    if (act) {
      const int r = run[warp][b] + below;
      int pos = -1;
      if (r < cnt[b]) {
        pos = off[b] + r;
        dpos[pos] = D;
      } else {
        atomicCAS(status, 0, 1 + STATUS_PLAN);
      }
      inv[(long)jj * n_ov + i * n_virt + a] = pos;
    }
    __syncwarp();
    if (act && below == 0) run[warp][b] += __popc(peers);
    __syncwarp();
  }
}

struct BinPos {
  int u0[SB_MAX_BINS + 1];  // first position of each bin
  int rank[SB_MAX_BINS];
};

// Skeleton weights w = zeta_k |d(D_u, w_skel[b][g])| of every position u and
// slot g < rmax (zero for padding, D = 0, and for slots past the bin's rank),
// as a 31-bit mantissa and exponent: w = wm 2^(ew - 31), wx = wm | ew << 32.
__global__ void __launch_bounds__(256) wskel_kernel(int Kt, int rmax, int nb, BinPos bp, const double* dpos,
                                                    const double* skel_om, double zeta_k, unsigned long long* wx,
                                                    int16_t* ewx) {
  const long total = (long)rmax * Kt;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int g = (int)(idx / Kt), u = (int)(idx - (long)g * Kt);
    int b = 0;
    while (b + 1 < nb && bp.u0[b + 1] <= u) ++b;
    unsigned long long out = (unsigned long long)(uint32_t)(-2000) << 32;
    const double D = dpos[u];
    if (g < bp.rank[b] && D > 0.0) {
      const double om = skel_om[b * rmax + g];
      const double w = zeta_k * (4.0 * D / (D * D + om * om));
      const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
      const int E = (int)((bits >> 52) & 0x7ff);
      if (E) {
        unsigned long long m = (((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) + (1ull << 21)) >> 22;
        int ee = E - 1022;
        if (m >> 31) {
          m >>= 1;
          ++ee;
        }
        out = m | ((unsigned long long)(uint32_t)ee << 32);
      }
    }
    wx[idx] = out;
    ewx[idx] = (int16_t)(int)(uint32_t)(out >> 32);
  }
}

// c_fix = round(c 2^(30 - eC)) of one FP64 value (eC: the row's exponent).
__device__ __forceinline__ int fix_of(unsigned long long cb, int eC) {
  const int Ec = (int)((cb >> 52) & 0x7ff);
  if (Ec == 0) return 0;
  const int sh = 1045 - Ec + eC;  // >= 23 since eC >= Ec - 1022
  if (sh >= 64) return 0;
  const unsigned long long mant = (cb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int m = (int)((mant + (1ull << (sh - 1))) >> sh);
  return (cb >> 63) ? -m : m;
}

// Fixed-point C in bin order: C read in its natural order (coalesced, a k-pair
// and t range per block, 8 rows of a warp each), each value written to its
// bin-order position (a row's values of one bin are contiguous there).  Rows
// N..Npad-1 are written as zeros; padding positions are zeroed by
// erow_bin_kernel.
__global__ void __launch_bounds__(256) cfix_scatter_kernel(int cplx, int N, int Npad, int n_ov, int Kr, int TP,
                                                           const double* const* C, const int* inv, const int* eCraw,
                                                           int* cfix) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = blockIdx.x * 8 + warp;
  if (P >= Npad) return;
  const int j = blockIdx.y / TP, tp = blockIdx.y - j * TP;
  const int t0 = (int)((long)tp * n_ov / TP), t1 = (int)((long)(tp + 1) * n_ov / TP);
  const int rc = P < N ? eCraw[P] : 0;
  const int eC = rc ? rc - 1022 : -2000;
  const int* invj = inv + (long)j * n_ov;
  int* out = cfix + (long)P * Kr;
  for (int t = t0 + lane; t < t1; t += 32) {
    const int pos = invj[t];
    if (pos < 0) continue;
    if (cplx) {
      int2 v = make_int2(0, 0);
      if (P < N) {
        const ulonglong2 x = reinterpret_cast<const ulonglong2*>(C[j])[(long)P * n_ov + t];
        v = make_int2(fix_of(x.x, eC), fix_of(x.y, eC));
      }
      *reinterpret_cast<int2*>(out + 2 * (long)pos) = v;
    } else {
      int v = 0;
      if (P < N) v = fix_of(reinterpret_cast<const unsigned long long*>(C[j])[(long)P * n_ov + t], eC);
      out[pos] = v;
    }
  }
}

// Raw row maxima of the weighted operand per (bin, skeleton slot) from the
// fixed-point values: |c_fix| < 2^bitlen, |w| < 2^ee, so
// raw = max (bitlen + ee) + eC + 2014 bounds |c w| < 2^(raw - 2044) for the
// values the slicing actually converts (the convention of the per-frequency
// path, where raw = exponent field of c + ee + 1022).  Block: EROW_BIN_ROWS
// rows (each warp several) x one part (a position range inside one bin); the
// part's weight exponents are staged in shared memory once for all its rows
// (slot 0's exponent is -2000 exactly at padding positions, which are zeroed
// here).
constexpr int EROW_BIN_ROWS = 64;
constexpr int EROW_ILP = 4;
template <int MR>  // skeletons per bin at most (register array size)
__global__ void __launch_bounds__(256) erow_bin_kernel(int cplx, int Npad, int Kr, int Kt, int rmax,
                                                       const int* parts, const int* rankb, const int* eCraw,
                                                       const int16_t* ewx, int* cfix, int* eAraw) {
  extern __shared__ int16_t ees[];  // [R][part length]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = parts[3 * blockIdx.y], u0 = parts[3 * blockIdx.y + 1], u1 = parts[3 * blockIdx.y + 2];
  const int len = u1 - u0;
  const int R = rankb[b];
  // positions and parts are multiples of 8, Kt too: 16-byte copies of the exponents
  const int len8 = len >> 3;
  for (int i = threadIdx.x; i < R * len8; i += blockDim.x) {
    const int g = i / len8, c = i - g * len8;
    *reinterpret_cast<uint4*>(ees + g * len + 8 * c) =
        __ldg(reinterpret_cast<const uint4*>(ewx + (long)g * Kt + u0) + c);
  }
  __syncthreads();
  for (int rr = 0; rr < EROW_BIN_ROWS / 8; ++rr) {
    const int P = blockIdx.x * EROW_BIN_ROWS + rr * 8 + warp;
    if (P >= Npad) break;
    int m[MR];
#pragma unroll
    for (int g = 0; g < MR; ++g) m[g] = -100000;
    int* row = cfix + (long)P * Kr;
    // EROW_ILP positions per lane per step: their loads are issued together
    for (int ub = 0; ub < len; ub += 32 * EROW_ILP) {
      int av[EROW_ILP];
#pragma unroll
      for (int k = 0; k < EROW_ILP; ++k) {
        const int uu = ub + k * 32 + lane;
        av[k] = 0;
        if (uu < len && ees[uu] != -2000) {
          const long u = u0 + uu;
          if (cplx) {
            const int2 v = *reinterpret_cast<const int2*>(row + 2 * u);
            av[k] = max(abs(v.x), abs(v.y));
          } else {
            av[k] = abs(row[u]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < EROW_ILP; ++k) {
        const int uu = ub + k * 32 + lane;
        if (uu >= len) break;
        if (ees[uu] == -2000) {  // padding position
          const long u = u0 + uu;
          if (cplx)
            *reinterpret_cast<int2*>(row + 2 * u) = make_int2(0, 0);
          else
            row[u] = 0;
          continue;
        }
        if (av[k] == 0) continue;
        const int bitlen = 32 - __clz(av[k]);
#pragma unroll
        for (int g = 0; g < MR; ++g) {
          if (g >= R) break;
          m[g] = max(m[g], bitlen + (int)ees[g * len + uu]);
        }
      }
    }
    const int rc = eCraw[P];
    if (!rc) continue;  // an all-zero row: no weighted contributions
    const int eC = rc - 1022;
#pragma unroll
    for (int g = 0; g < MR; ++g) {
      if (g >= R) break;
      const int r = __reduce_max_sync(0xffffffffu, m[g]);
      if (lane == 0 && r > -100000) atomicMax(eAraw + ((long)b * rmax + g) * Npad + P, max(0, r + eC + 2014));
    }
  }
}

__global__ void __launch_bounds__(256, 2) slice_bin_kernel(SliceBinArgs a) {
  const long total = (long)a.Npad * a.n_kb;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    if (a.cplx)
      slice_unit_bin<true>(a, idx);
    else
      slice_unit_bin<false>(a, idx);
  }
}

// chi0(w) for every frequency from the partials of every (bin, skeleton):
// one thread per element of a lower tile.  The combination sum_{b,r} coef x
// (n_w x sum_b rank_b multiply-adds per element) runs in float-float
// arithmetic on the FP32 pipe (GB300's FP64 pipe is 1/58 of it): coef is held
// as an unevaluated sum of two floats, each product is formed exactly by
// Dekker's TwoProd (fmaf), and sums use Knuth's TwoSum; about 2^-44 relative,
// far below the split-precision error of the partials.  Frequencies are
// taken in groups of at most RED_WG along grid y (registers).
struct RedBin {
  int cplx, N, Npad, n_tiles, nb, rmax, n_w, G;  // G: skeleton slots per round
  int rank[SB_MAX_BINS], nks[SB_MAX_BINS];
  long base[SB_MAX_BINS];  // item index of bin b's first round
  const float* part;
  const int* eAraw;
  const int* eCraw;
  const double* coef;  // [nb][rmax][n_w]
  double* chi;         // [n_w][N][N]
  int wg;              // frequencies per group (grid y = groups)
};
constexpr int RED_WG = 10;

// (h, l) += a + b (a, b: a float-float product), Knuth TwoSum then renormalise.
__device__ __forceinline__ void ff_acc(float& h, float& l, float ph, float pl) {
  const float s = h + ph;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (ph - bb);
  const float t = e + pl + l;
  h = s + t;
  l = t - (h - s);
}

__global__ void __launch_bounds__(256, 2) reduce_bin_kernel(const __grid_constant__ RedBin rb) {
  extern __shared__ float2 cs[];  // coefficients as (hi, lo) floats
  const int ncoef = rb.nb * rb.rmax * rb.n_w;
  for (int i = threadIdx.x; i < ncoef; i += blockDim.x) {
    const double c = rb.coef[i];
    const float h = (float)c;
    cs[i] = make_float2(h, (float)(c - (double)h));
  }
  __syncthreads();
  const int ncols = rb.cplx ? 64 : 128;
  const int per_tile = 128 * ncols / 256;
  const int tile = blockIdx.x / per_tile;
  const int e = (blockIdx.x - tile * per_tile) * 256 + threadIdx.x;
  const int r = e / ncols, c = e - (e / ncols) * ncols;
  int I, J;
  tile_ij(rb.cplx, tile, I, J);
  const int P = I * 128 + r, Q = J * ncols + c;
  if (P >= rb.N || Q >= rb.N || Q > P) return;
  const int w0 = blockIdx.y * rb.wg, nw = min(rb.wg, rb.n_w - w0);
  float rh[RED_WG], rl[RED_WG], ih[RED_WG], il[RED_WG];
#pragma unroll
  for (int w = 0; w < RED_WG; ++w) rh[w] = rl[w] = ih[w] = il[w] = 0.f;
  const int rq = rb.eCraw[Q];
  const int eCQ = rq ? rq - 1022 : -2000;
  for (int b = 0; b < rb.nb; ++b) {
    for (int g = 0; g < rb.rank[b]; ++g) {
      const int ra = rb.eAraw[((long)b * rb.rmax + g) * rb.Npad + P];
      if (ra <= 0 || rq == 0) continue;  // a zero row or column: no contribution
      const int g0 = g / rb.G * rb.G, Gs = min(rb.G, rb.rank[b] - g0), gl = g - g0;
      const long it0 = rb.base[b] + (long)g0 * rb.nks[b] * rb.n_tiles;
      // x = sum over the split-K partials of (hi + lo), as a float-float pair
      float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
      for (int ks = 0; ks < rb.nks[b]; ++ks) {
        const long item = it0 + ((long)ks * Gs + gl) * rb.n_tiles + tile;
        const float* pp = rb.part + item * 2 * 128 * 128 + (long)r * 128;
        ff_acc(xh, xl, pp[c], pp[128 * 128 + c]);
        if (rb.cplx) ff_acc(yh, yl, pp[64 + c], pp[128 * 128 + 64 + c]);
      }
      // scale 2^(eA + eC + 1 - 14) with the sign of chi = -sum conj(a) c (exact)
      const int sh = (ra - 2044 + 1) + eCQ + 1 - 14;
      xh = -ldexpf(xh, sh);
      xl = -ldexpf(xl, sh);
      yh = -ldexpf(yh, sh);
      yl = -ldexpf(yl, sh);
      const float2* cf = cs + ((long)b * rb.rmax + g) * rb.n_w + w0;
#pragma unroll
      for (int w = 0; w < RED_WG; ++w) {
        if (w >= nw) break;
        const float2 k = cf[w];
        float ph = k.x * xh;
        float pl = fmaf(k.x, xh, -ph) + fmaf(k.x, xl, k.y * xh);
        ff_acc(rh[w], rl[w], ph, pl);
        if (rb.cplx) {
          ph = k.x * yh;
          pl = fmaf(k.x, yh, -ph) + fmaf(k.x, yl, k.y * yh);
          ff_acc(ih[w], il[w], ph, pl);
        }
      }
    }
  }
  const long NN = (long)rb.N * rb.N;
#pragma unroll
  for (int w = 0; w < RED_WG; ++w) {
    if (w >= nw) break;
    const double re = (double)rh[w] + (double)rl[w];
    if (rb.cplx) {
      double2* out = reinterpret_cast<double2*>(rb.chi) + (long)(w0 + w) * NN;
      const double im = P == Q ? 0.0 : (double)ih[w] + (double)il[w];
      out[(long)P * rb.N + Q] = make_double2(re, im);
      if (P != Q) out[(long)Q * rb.N + P] = make_double2(re, -im);
    } else {
      double* out = rb.chi + (long)(w0 + w) * NN;
      out[(long)P * rb.N + Q] = re;
      if (P != Q) out[(long)Q * rb.N + P] = re;
    }
  }
}

// ------------------------------------------------------------ host side --

// Workspace of the frequency-batched path: per-q regions (the q's tables,
// fixed-point C, digit planes of C, split-K partials) and weighted-operand
// buffers (G skeleton slots of every bin).  Pipelined: two of each, so that
// every tensor-core launch (a round of one q) writes the next round's weighted
// planes in its slicer warps while the next q's preparation sits in the other
// region; otherwise one of each and standalone slicing launches.
struct BinLayout {
  int Npad, Kt, Kr, n_kb, nb, rmax, G, n_tiles, n_parts, meta_ints, nreg;
  long items;  // partial items of one q (sum over bins of rank x split-K cap x tiles)
  size_t meta, inv, dpos, wx, ewx, eC, eA, cfix, SC, part, qreg, abuf, total;
};

BinLayout bin_layout_g(const BatchGeom& g, const FreqPlan& p, int Kt_max, int n_parts_max, int s, int G, int nreg,
                       int sms) {
  BinLayout L{};
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  L.Npad = (g.n_aux + 127) / 128 * 128;
  L.Kt = Kt_max;
  L.Kr = g.cplx ? 2 * Kt_max : Kt_max;
  L.n_kb = L.Kr / KB;
  L.nb = p.n_bins;
  L.rmax = p.rmax;
  L.G = G;
  L.nreg = nreg;
  L.n_parts = n_parts_max;
  const int nbk = L.Npad / 128;
  L.n_tiles = g.cplx ? nbk * (nbk + 1) : nbk * (nbk + 1) / 2;
  const size_t per_slot = (size_t)s * L.Npad * L.Kr * 2;  // every bin's weighted planes of one slot
  // split-K cap per bin: enough items to fill the GPU (the partial buffer is sized for it)
  long items = 0;
  const int chunks = (L.n_kb + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
  for (int b = 0; b < L.nb; ++b) {
    const int Gb = std::min(G, p.rank[b]);
    const int cap = std::max(1, std::min(chunks, (4 * sms + Gb * L.n_tiles - 1) / std::max(1, Gb * L.n_tiles)));
    items += (long)p.rank[b] * cap * L.n_tiles;
  }
  L.items = items;
  L.meta_ints = 2 * g.n_k * g.n_occ * L.nb + 3 * L.n_parts + SB_MAX_BINS;
  L.meta = al(sizeof(int) * (size_t)L.meta_ints + 64) + al(sizeof(double) * (size_t)L.nb * L.rmax * (1 + g.n_w));
  L.inv = al(sizeof(int) * (size_t)g.n_k * g.n_ov);
  L.dpos = al(sizeof(double) * (size_t)L.Kt);
  L.wx = al(sizeof(unsigned long long) * (size_t)L.rmax * L.Kt);
  L.ewx = al(sizeof(int16_t) * (size_t)L.rmax * L.Kt);
  L.eC = al(sizeof(int) * (size_t)L.Npad);
  L.eA = al(sizeof(int) * (size_t)L.nb * L.rmax * L.Npad);
  L.cfix = al(sizeof(int) * (size_t)L.Npad * L.Kr);
  L.SC = al(per_slot * (g.cplx ? 2 : 1));
  L.part = al(sizeof(float) * 2 * 128 * 128 * (size_t)items);
  L.qreg = L.meta + L.inv + L.dpos + L.wx + L.ewx + L.eC + L.eA + L.cfix + L.SC + L.part;
  L.abuf = al(per_slot * G);
  L.total = 1024 + nreg * (L.qreg + L.abuf);
  return L;
}

// Within `budget`: pipelined with every skeleton in one round per q; else one
// region with every skeleton in one round; else one region with the largest
// round that fits (G = 1 when nothing fits: the caller reports the shortfall).
// Pipelining several rounds of one q was measured slower on the slab job (the
// slicer warps' stores pull the power-capped clock down by more than the
// standalone slicing costs), so it is not used.
BinLayout bin_layout(const BatchGeom& g, const FreqPlan& p, int Kt_max, int n_parts_max, int s, size_t budget,
                     int sms) {
  for (int nreg = 2; nreg >= 1; --nreg) {
    const BinLayout L = bin_layout_g(g, p, Kt_max, n_parts_max, s, p.rmax, nreg, sms);
    if (L.total <= budget) return L;
  }
  for (int G = p.rmax - 1; G >= 1; --G) {
    const BinLayout L = bin_layout_g(g, p, Kt_max, n_parts_max, s, G, 1, sms);
    if (L.total <= budget) return L;
  }
  return bin_layout_g(g, p, Kt_max, n_parts_max, s, 1, 1, sms);
}

// One q's region: tables, exponents, fixed-point C, digit planes of C, partials.
struct BinRegion {
  int* meta_i;     // rowtab [2][n_k n_occ nb] | parts [n_parts][3] | rank [16]
  double* meta_d;  // skel_om [nb][rmax] | coef [nb][rmax][n_w]
  int *inv, *eC, *eA, *cfix;
  double* dpos;
  unsigned long long* wx;
  int16_t* ewx;
  uint16_t* SC;
  float* part;
};

BinRegion carve_bin(char* p, const BinLayout& L) {
  BinRegion r;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  r.meta_i = (int*)p;
  r.meta_d = (double*)(p + al(sizeof(int) * (size_t)L.meta_ints + 64));
  p += L.meta;
  r.inv = (int*)p;
  p += L.inv;
  r.dpos = (double*)p;
  p += L.dpos;
  r.wx = (unsigned long long*)p;
  p += L.wx;
  r.ewx = (int16_t*)p;
  p += L.ewx;
  r.eC = (int*)p;
  p += L.eC;
  r.eA = (int*)p;
  p += L.eA;
  r.cfix = (int*)p;
  p += L.cfix;
  r.SC = (uint16_t*)p;
  p += L.SC;
  r.part = (float*)p;
  return r;
}

constexpr int BIN_PREP_LAUNCHES = 6;  // ecrow, perm, wskel, cfix_scatter, erow_bin, slice of C

// Region R as q's kernels see it: the tables read in place when the job's
// copy of them is on the device already.
BinRegion region_of(const BinRegion& R, const MixedBinQ& q) {
  BinRegion r = R;
  if (q.host->dmeta_i && q.host->dmeta_d) {
    r.meta_i = const_cast<int*>(q.host->dmeta_i);
    r.meta_d = const_cast<double*>(q.host->dmeta_d);
  }
  return r;
}

// Steps 1-6 for one q into region R, after copying its table image there.
cudaError_t bin_prep(const BinRegion& R, const BinLayout& L, const MixedBinQ& q, const FreqPlan& p, int s, int sms,
                     cudaStream_t st) {
  const BatchGeom& g = q.g;
  const BinQHost& h = *q.host;
  cudaError_t e = cudaSuccess;
  if (R.meta_i != h.dmeta_i) {
    e = cudaMemcpyAsync(R.meta_i, h.meta_i, sizeof(int) * h.n_meta_i, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(R.meta_d, h.meta_d, sizeof(double) * h.n_meta_d, cudaMemcpyHostToDevice, st);
    if (e) return e;
  }
  if ((e = cudaMemsetAsync(R.dpos, 0, sizeof(double) * (size_t)h.Kt, st))) return e;
  if ((e = cudaMemsetAsync(R.eC, 0, sizeof(int) * (size_t)L.Npad, st))) return e;
  if ((e = cudaMemsetAsync(R.eA, 0, sizeof(int) * (size_t)L.nb * L.rmax * L.Npad, st))) return e;
  const int TP = g.n_k >= 8 ? 1 : (8 + g.n_k - 1) / g.n_k;
  ecrow_kernel<<<dim3((unsigned)((g.n_aux + 7) / 8), (unsigned)(g.n_k * TP)), 256, 0, st>>>(g.cplx, g.n_aux, g.n_ov,
                                                                                          TP, q.Cptrs, R.eC);
  BinEdges be{};
  for (int b = 0; b + 1 < p.n_bins; ++b) be.edge[b] = p.edges[b];
  const long nrow = (long)g.n_k * g.n_occ;
  perm_kernel<<<(unsigned)((nrow + 7) / 8), 256, 0, st>>>(g.n_k, g.n_occ, g.n_virt, p.n_bins, be, q.eps_occ,
                                                          q.eps_virt, q.kidx, q.kqidx, R.meta_i, R.inv, R.dpos,
                                                          q.status);
  BinPos bp{};
  for (int b = 0; b <= p.n_bins; ++b) bp.u0[b] = h.tb0[b];
  for (int b = p.n_bins + 1; b <= SB_MAX_BINS; ++b) bp.u0[b] = h.Kt;
  for (int b = 0; b < p.n_bins; ++b) bp.rank[b] = p.rank[b];
  const long nw = (long)L.rmax * h.Kt;
  wskel_kernel<<<(unsigned)std::min<long>((nw + 255) / 256, (long)sms * 16), 256, 0, st>>>(
      h.Kt, L.rmax, p.n_bins, bp, R.dpos, R.meta_d, q.zeta_k, R.wx, R.ewx);
  cfix_scatter_kernel<<<dim3((unsigned)(L.Npad / 8), (unsigned)(g.n_k * TP)), 256, 0, st>>>(
      g.cplx, g.n_aux, L.Npad, g.n_ov, h.Kr, TP, q.Cptrs, R.inv, R.eC, R.cfix);
  const int n_parts = h.n_parts;
  const int* parts = R.meta_i + 2 * nrow * p.n_bins;
  const int* rankb = parts + 3 * n_parts;
  const dim3 eg((unsigned)((L.Npad + EROW_BIN_ROWS - 1) / EROW_BIN_ROWS), (unsigned)n_parts);
  const size_t esm = sizeof(int16_t) * (size_t)L.rmax * FREQ_PART;
  if (L.rmax <= 8)
    erow_bin_kernel<8><<<eg, 256, esm, st>>>(g.cplx, L.Npad, h.Kr, h.Kt, L.rmax, parts, rankb, R.eC, R.ewx, R.cfix,
                                             R.eA);
  else if (L.rmax <= 16)
    erow_bin_kernel<16><<<eg, 256, esm, st>>>(g.cplx, L.Npad, h.Kr, h.Kt, L.rmax, parts, rankb, R.eC, R.ewx,
                                              R.cfix, R.eA);
  else
    erow_bin_kernel<32><<<eg, 256, esm, st>>>(g.cplx, L.Npad, h.Kr, h.Kt, L.rmax, parts, rankb, R.eC, R.ewx,
                                              R.cfix, R.eA);
  // digits of C (the B operand) in bin order
  SliceArgs sc{g.cplx, L.Npad, g.n_ov, h.Kt, h.Kr, s, g.n_w, 0, 1, g.cplx ? 2 : 1, R.cfix, nullptr,
               nullptr, nullptr, R.SC};
  const long tg = (long)L.Npad * (h.Kr / 16);
  launch_slice(g.cplx, (unsigned)std::min<long>((tg + 255) / 256, (long)sms * 32), st, sc);
  return cudaGetLastError();
}

// Weighted planes of round k (slots [k G, k G + G) of every bin) of one q into A.
SliceBinArgs bin_slice_args(const BinRegion& R, uint16_t* A, const BinLayout& L, const MixedBinQ& q,
                            const FreqPlan& p, int s, int k) {
  const BinQHost& h = *q.host;
  SliceBinArgs a{};
  a.cplx = q.g.cplx;
  a.Npad = L.Npad;
  a.Kr = h.Kr;
  a.s = s;
  a.n_kb = h.Kr / KB;
  a.nb = p.n_bins;
  a.g0 = k * L.G;
  a.rmax = L.rmax;
  a.Kt = h.Kt;
  a.cfix = R.cfix;
  a.eC = R.eC;
  a.wx = R.wx;
  a.eAraw = R.eA;
  a.S = A;
  const long nI = L.Npad / 128;
  long off = 0;
  const int tpk = q.g.cplx ? 8 : 16;
  for (int b = 0; b < SB_MAX_BINS; ++b) {
    const bool in = b < p.n_bins;
    a.kb0[b] = in ? h.tb0[b] / tpk : a.n_kb;
    a.G[b] = in ? std::max(0, std::min(L.G, p.rank[b] - a.g0)) : 0;
    a.aoff[b] = off;
    if (in) off += (long)a.G[b] * nI * ((h.tb0[b + 1] - h.tb0[b]) / tpk) * s * 2048;
  }
  a.kb0[SB_MAX_BINS] = a.n_kb;
  return a;
}

void launch_slice_bin(const SliceBinArgs& sa, int Npad, int sms, cudaStream_t st) {
  const long tg = (long)Npad * sa.n_kb;
  slice_bin_kernel<<<(unsigned)std::min<long>((tg + 255) / 256, (long)sms * 32), 256, 0, st>>>(sa);
}

// Split-K depth of every bin for q (fixed over its rounds): the cost model of
// the per-frequency path over the first round's segments, or the recorded
// autotuner choice for this shape class.
void bin_splits(const BinLayout& L, const MixedBinQ& q, const FreqPlan& p, int s, int sms, int* nks) {
  const BinQHost& h = *q.host;
  const int tpk = q.g.cplx ? 8 : 16;
  std::vector<SegShape> shp;
  std::vector<int> who;
  const int chunks_all = (L.n_kb + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
  for (int b = 0; b < p.n_bins; ++b) {
    const int nkb = (h.tb0[b + 1] - h.tb0[b]) / tpk;
    nks[b] = 1;
    if (nkb == 0) continue;
    const int chunks = (nkb + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
    const int Gb = std::min(L.G, p.rank[b]);
    const int cap = std::max(1, std::min(chunks_all, (4 * sms + Gb * L.n_tiles - 1) / std::max(1, Gb * L.n_tiles)));
    shp.push_back(SegShape{chunks, Gb, L.n_tiles, std::min(cap, chunks)});
    who.push_back(b);
  }
  if (shp.empty()) return;
  int Lc = autotune_lookup(round_key(shp, s) ^ 0x5bd1e995ull);
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
  for (size_t i = 0; i < who.size(); ++i) nks[who[i]] = pl.nks[i];
}

// The tensor-core launch of round k of q (segments: the bins with slots in it).
int bin_tc_params(const BinRegion& R, const uint16_t* A, const BinLayout& L, const MixedBinQ& q, const FreqPlan& p,
                  int s, int k, const int* nks, const long* base, int* err, TcParams& tp) {
  const BinQHost& h = *q.host;
  const int tpk = q.g.cplx ? 8 : 16;
  memset(&tp, 0, sizeof tp);
  tp.s = s;
  tp.kb_per_chunk = KB_PER_CHUNK;
  tp.drop_item = mixed_test_drop_take();
  tp.err = err;
  tp.grp_mask = group_mask(s);
  const SliceBinArgs sa = bin_slice_args(R, const_cast<uint16_t*>(A), L, q, p, s, k);
  int items = 0;
  for (int b = 0; b < p.n_bins; ++b) {
    const int nkb = (h.tb0[b + 1] - h.tb0[b]) / tpk;
    const int Gs = sa.G[b];
    if (Gs <= 0 || nkb == 0) continue;
    const int chunks = (nkb + KB_PER_CHUNK - 1) / KB_PER_CHUNK;
    const int cps = (chunks + nks[b] - 1) / nks[b];
    TcSeg& S = tp.seg[tp.n_segs++];
    S.A = A + sa.aoff[b];
    S.B = R.SC;
    S.nI = L.Npad / 128;
    S.part = R.part + (base[b] + (long)sa.g0 * nks[b] * L.n_tiles) * 2 * 128 * 128;
    S.cplx = q.g.cplx;
    S.G = Gs;
    S.n_tiles = L.n_tiles;
    S.n_ksplit = nks[b];
    S.kb_per_split = cps * KB_PER_CHUNK;
    S.n_kb = nkb;
    S.kb_off = sa.kb0[b];
    S.ldb = sa.n_kb;
    S.item0 = items;
    items += Gs * L.n_tiles * nks[b];
  }
  tp.n_items = items;
  return items;
}

}  // namespace

size_t binned_workspace_bytes(const BatchGeom& g, const FreqPlan& p, int Kt_max, int n_parts_max, int n_slices,
                              size_t budget, int* slots, int* regions) {
  const BinLayout L = bin_layout(g, p, Kt_max, n_parts_max, n_slices, budget, num_sms());
  if (slots) *slots = L.G;
  if (regions) *regions = L.nreg;
  return L.total;
}

// chi0 of n q (one geometry) through the frequency-batched plan.  The launches
// run as a sequence of units (q, round); with the pipelined layout each
// tensor-core launch writes the next unit's weighted planes in its slicer
// warps (the first unit's are a launch of their own), and the next q's
// preparation runs before the last launch of the current q.
cudaError_t launch_chi0_binned(const MixedBinQ* qs, int n, const FreqPlan& p, int s, void* work, size_t work_bytes,
                               int* status, uint64_t* n_launch, cudaStream_t st, const LaunchHook* hook) {
  auto hb = [&]() {
    if (hook) hook->begin(hook->user, st);
  };
  auto he = [&](int cls, int nk) {
    if (hook) hook->end(hook->user, st, cls, nk);
  };
  if (n <= 0) return cudaSuccess;
  if (s < 2 || s > MAX_S || p.n_bins <= 0 || p.rmax > BIN_MAX_RANK) return cudaErrorInvalidValue;
  if ((size_t)p.n_bins * p.rmax * qs[0].g.n_w * sizeof(double) > 48 * 1024) return cudaErrorInvalidValue;
  const int sms = num_sms();
  if (cudaError_t ea = tc_smem_attr()) return ea;
  {
    static std::once_flag once;
    static cudaError_t ea2 = cudaSuccess;
    std::call_once(once, [] {
      const int bytes = (int)(sizeof(int16_t) * BIN_MAX_RANK * FREQ_PART);
      ea2 = cudaFuncSetAttribute(erow_bin_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (ea2 == cudaSuccess)
        ea2 = cudaFuncSetAttribute(erow_bin_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (ea2 == cudaSuccess)
        ea2 = cudaFuncSetAttribute(erow_bin_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
    if (ea2) return ea2;
  }
  int Kt_max = 0, np_max = 0;
  for (int i = 0; i < n; ++i) {
    Kt_max = std::max(Kt_max, qs[i].host->Kt);
    np_max = std::max(np_max, qs[i].host->n_parts);
  }
  const BinLayout L = bin_layout(qs[0].g, p, Kt_max, np_max, s, work_bytes, sms);
  if (L.total > work_bytes) return cudaErrorMemoryAllocation;
  const bool pipe = L.nreg == 2;
  char* base = (char*)work;
  int* err = (int*)base;
  BinRegion R[2];
  uint16_t* AB[2];
  for (int r = 0; r < L.nreg; ++r) {
    R[r] = carve_bin(base + 1024 + r * L.qreg, L);
    AB[r] = (uint16_t*)(base + 1024 + L.nreg * L.qreg + r * L.abuf);
  }
  if (!pipe) {
    R[1] = R[0];
    AB[1] = AB[0];
  }
  uint64_t nl = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return e;
  const int rounds = (p.rmax + L.G - 1) / L.G;
  const int n_units = n * rounds;
  // the first q's preparation and the first unit's weighted planes
  hb();
  if ((e = bin_prep(region_of(R[0], qs[0]), L, qs[0], p, s, sms, st))) return e;
  launch_slice_bin(bin_slice_args(region_of(R[0], qs[0]), AB[0], L, qs[0], p, s, 0), L.Npad, sms, st);
  he(RPA_K_SLICE, BIN_PREP_LAUNCHES + 1);
  nl += BIN_PREP_LAUNCHES + 1;
  int nks[SB_MAX_BINS];
  long bbase[SB_MAX_BINS];
  for (int u = 0; u < n_units; ++u) {
    const int i = u / rounds, k = u - i * rounds;
    const MixedBinQ& q = qs[i];
    const BinRegion C = region_of(R[i & 1], q);
    uint16_t* A = AB[u & 1];
    if (!pipe && u > 0) {  // one region and one buffer: preparation and slicing as launches of their own
      hb();
      int nk = 1;
      if (k == 0) {
        if ((e = bin_prep(C, L, q, p, s, sms, st))) return e;
        nk += BIN_PREP_LAUNCHES;
      }
      launch_slice_bin(bin_slice_args(C, A, L, q, p, s, k), L.Npad, sms, st);
      he(RPA_K_SLICE, nk);
      nl += nk;
    }
    if (k == 0) {
      bin_splits(L, q, p, s, sms, nks);
      long items = 0;
      for (int b = 0; b < p.n_bins; ++b) {
        bbase[b] = items;
        items += (long)p.rank[b] * nks[b] * L.n_tiles;
      }
      if (items > L.items) return cudaErrorInvalidValue;
    }
    const bool has_next = pipe && u + 1 < n_units;
    const int i2 = (u + 1) / rounds, k2 = (u + 1) - i2 * rounds;
    if (has_next && i2 != i) {  // the next q's preparation in the other region
      hb();
      if ((e = bin_prep(region_of(R[i2 & 1], qs[i2]), L, qs[i2], p, s, sms, st))) return e;
      he(RPA_K_SLICE, BIN_PREP_LAUNCHES);
      nl += BIN_PREP_LAUNCHES;
    }
    TcParams tp;
    const int n_items = bin_tc_params(C, A, L, q, p, s, k, nks, bbase, err, tp);
    if (has_next) {
      tp.side_on = 2;
      tp.sideb = bin_slice_args(region_of(R[i2 & 1], qs[i2]), AB[(u + 1) & 1], L, qs[i2], p, s, k2);
    }
    if (n_items > 0) {
      hb();
      launch_tc(s, std::min(n_items, sms), TC_SMEM, st, tp);
      he(RPA_K_CHI0, 1);
      ++nl;
    } else if (has_next) {  // nothing to contract: the next unit's planes standalone
      launch_slice_bin(tp.sideb, L.Npad, sms, st);
      ++nl;
    }
    if (k == rounds - 1) {
      RedBin rb{};
      rb.cplx = q.g.cplx;
      rb.N = q.g.n_aux;
      rb.Npad = L.Npad;
      rb.n_tiles = L.n_tiles;
      rb.nb = p.n_bins;
      rb.rmax = L.rmax;
      rb.n_w = q.g.n_w;
      rb.G = L.G;
      for (int b = 0; b < p.n_bins; ++b) {
        rb.rank[b] = (q.host->tb0[b + 1] > q.host->tb0[b]) ? p.rank[b] : 0;
        rb.nks[b] = nks[b];
        rb.base[b] = bbase[b];
      }
      rb.part = C.part;
      rb.eAraw = C.eA;
      rb.eCraw = C.eC;
      rb.coef = C.meta_d + (size_t)p.n_bins * L.rmax;
      rb.chi = q.chi;
      const int per_tile = 128 * (q.g.cplx ? 64 : 128) / 256;
      const int n_groups = (q.g.n_w + RED_WG - 1) / RED_WG;
      rb.wg = (q.g.n_w + n_groups - 1) / n_groups;
      hb();
      reduce_bin_kernel<<<dim3((unsigned)(L.n_tiles * per_tile), (unsigned)n_groups), 256,
                          sizeof(float2) * (size_t)p.n_bins * L.rmax * q.g.n_w, st>>>(rb);
      he(RPA_K_CHI0_RED, 1);
      ++nl;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (status) {
    err_merge_kernel<<<1, 32, 0, st>>>(err, status);
    ++nl;
  }
  if (n_launch) *n_launch = nl;
  return cudaSuccess;
}

}  // namespace rpa
