// BF16 digit planes of the split-precision chi0 operands: the per-unit
// slicing code, shared by the standalone slicing kernel and the spare warps of
// the tensor-core kernel (which write the next q's weighted operand while the
// current q's MMAs run).
//
// A digit set is produced from an integer F (|F| <= 2^30):
//   F + 0x808080 = (d0 2^24) + (d1+128) 2^16 + (d2+128) 2^8 + (d3+128),
// each biased byte b is turned into the BF16 of (b - 128) 2^(-8i) by the
// exact float trick (2^23 + b) 2^(-8i) - (2^23 + 128) 2^(-8i) (one FFMA, no I2F).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpa {
namespace {

constexpr int MAX_S = 4;  // digit planes at most


struct SliceArgs {
  int cplx, Npad, n_ov, Ktot, Kr, s, n_w, w0, G, nxy;
  const int* cfix;       // [Npad][Kr]
  const int* eC;         // [Npad] exponent of c_fix
  const unsigned long long* wx;  // [n_k][n_w][n_ov] weights (mantissa | exponent << 32), null: weight 1
  const int* eA;         // [n_w][Npad] row exponents of A
  uint16_t* S;           // digit planes, blocked (see store_planes)
};

// One thread per (row, 16 real values); it loops over the G frequencies of the
// launch (the 16 fixed-point values of C are loaded once).  With wm == null
// the digits of C itself are written (X and, for complex data, Y = (im, -re)).
// Digit planes are stored in the order the tensor-core kernel consumes them,
// so that one stage of operand data is a single contiguous 16 KB copy:
//   weighted A: [g][I = P/128][kb][plane][m-core 16][k-core 2][8 rows][8 values]
//   C (B side): [J][kb][plane][n-core 16][k-core 2][8 rows][8 values]
// with J = P/64 for complex data (n-cores 0-7: X rows, 8-15: Y rows) and
// J = P/128 for real data.  A 4 KB plane block is the no-swizzle K-major
// core-matrix layout of a 128 x 16 BF16 operand tile (core matrix = 8 rows x
// 16 bytes, K-adjacent cores 128 B apart, row-adjacent cores 256 B apart).
__device__ __forceinline__ void store_core_rows(uint16_t* block, int row, const uint32_t (&v)[8]) {
  uint4* d0 = reinterpret_cast<uint4*>(block + (((row >> 3) * 2 + 0) * 8 + (row & 7)) * 8);
  uint4* d1 = reinterpret_cast<uint4*>(block + (((row >> 3) * 2 + 1) * 8 + (row & 7)) * 8);
  *d0 = make_uint4(v[0], v[1], v[2], v[3]);
  *d1 = make_uint4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void store_planes(const SliceArgs& a, int P, int kb, const uint32_t (&px)[MAX_S][8],
                                             const uint32_t (&py)[MAX_S][8]) {
  const long n_kb = a.Kr / 16;
  const int J = a.nxy == 2 ? (P >> 6) : (P >> 7);
  const int nrow = a.nxy == 2 ? (P & 63) : (P & 127);
#pragma unroll
  for (int i = 0; i < MAX_S; ++i) {
    if (i >= a.s) break;
    uint16_t* blk = a.S + (((long)J * n_kb + kb) * a.s + i) * 2048;
    store_core_rows(blk, nrow, px[i]);
    if (a.nxy == 2) store_core_rows(blk, 64 + nrow, py[i]);
  }
}

// X planes only (the weighted operand A has no Y part).
__device__ __forceinline__ void store_planes_x(const SliceArgs& a, int g, int P, int kb,
                                               const uint32_t (&px)[MAX_S][8]) {
  const long n_kb = a.Kr / 16;
  const long nI = a.Npad / 128;
#pragma unroll
  for (int i = 0; i < MAX_S; ++i) {
    if (i >= a.s) break;
    uint16_t* blk = a.S + ((((long)g * nI + (P >> 7)) * n_kb + kb) * a.s + i) * 2048;
    store_core_rows(blk, P & 127, px[i]);
  }
}


// BF16 digit i of a biased word G' = (F + 0x808080) ^ 2^31 (byte 3 - i holds
// d_i + 128) as FP32 bits: one byte permute builds 2^23 + b, one FFMA scales
// and removes the bias exactly.
template <int I>
__device__ __forceinline__ uint32_t digit_f(uint32_t Gp) {
  const uint32_t bits = __byte_perm(Gp, 0x4B000000u, 0x7540u | (3 - I));
  const float scale = __int_as_float((127 - 8 * I) << 23);
  return __float_as_uint(fmaf(__uint_as_float(bits), scale, -8388736.0f * scale));
}
__device__ __forceinline__ uint32_t biased(int F) { return (uint32_t)(F + 0x808080) ^ 0x80000000u; }

// X digit planes of two consecutive K values (F0 low half, F1 high half).
__device__ __forceinline__ void pair_x(int F0, int F1, int up, int s, uint32_t (&px)[MAX_S][8]) {
  const uint32_t G0 = biased(F0), G1 = biased(F1);
  px[0][up] = __byte_perm(digit_f<0>(G0), digit_f<0>(G1), 0x7632);
  px[1][up] = __byte_perm(digit_f<1>(G0), digit_f<1>(G1), 0x7632);
  if (s > 2) px[2][up] = __byte_perm(digit_f<2>(G0), digit_f<2>(G1), 0x7632);
  if (s > 3) px[3][up] = __byte_perm(digit_f<3>(G0), digit_f<3>(G1), 0x7632);
}
// X = (re, im) and Y = (im, -re) digit planes of one complex value.
template <int I>
__device__ __forceinline__ void cplx_xy(uint32_t Gre, uint32_t Gim, uint32_t& x, uint32_t& y) {
  const uint32_t fr = digit_f<I>(Gre), fi = digit_f<I>(Gim);
  x = __byte_perm(fr, fi, 0x7632);
  y = __byte_perm(fi, fr ^ 0x80000000u, 0x7632);
}

// F = round(c w 2^-sh) for |c w| < 2^61; sh >= 1 by construction of the row
// exponents (|F| <= 2^30); sh is clamped to 62, where the result is 0 anyway.
__device__ __forceinline__ int round_shift(int c, long long wm, int sh) {
  sh = min(max(sh, 1), 62);
  const long long pr = (long long)c * wm;
  return (int)((pr + (1ll << (sh - 1))) >> sh);
}

// One unit of the slicing: row P = idx mod Npad and K-block tg = idx / Npad;
// the weighted form runs the G frequencies of the launch (the 16 fixed-point
// values of C are loaded once), the unweighted one writes the digits of C.
template <bool CPLX, bool WEIGHTED>
__device__ __forceinline__ void slice_unit(const SliceArgs& a, long idx) {
  constexpr int tpg = CPLX ? 8 : 16;  // t per group of 16 real values
  const int P = (int)(idx % a.Npad);
  const int tg = (int)(idx / a.Npad);
  const int4* src = reinterpret_cast<const int4*>(a.cfix + (long)P * a.Kr + tg * 16);
  int cv[16];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int4 x = src[v];
    cv[4 * v] = x.x;
    cv[4 * v + 1] = x.y;
    cv[4 * v + 2] = x.z;
    cv[4 * v + 3] = x.w;
  }
  if constexpr (!WEIGHTED) {
    uint32_t px[MAX_S][8], py[MAX_S][8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      if constexpr (CPLX) {
        const uint32_t Gr = biased(cv[2 * v]), Gi = biased(cv[2 * v + 1]);
        cplx_xy<0>(Gr, Gi, px[0][v], py[0][v]);
        cplx_xy<1>(Gr, Gi, px[1][v], py[1][v]);
        cplx_xy<2>(Gr, Gi, px[2][v], py[2][v]);
        cplx_xy<3>(Gr, Gi, px[3][v], py[3][v]);
      } else {
        pair_x(cv[2 * v], cv[2 * v + 1], v, a.s, px);
      }
    }
    store_planes(a, P, tg, px, py);
    return;
  } else {
    // the group's t = t0 .. t0 + tpg - 1 as (k-point j, pair tt): one
    // division per group, then steps
    const int t0 = tg * tpg;
    const int j0 = t0 / a.n_ov, tt0 = t0 - j0 * a.n_ov;
    const int eC = a.eC[P];
    // (k-point, pair) offsets of the group's t, frequency-independent
    long off[tpg];
    {
      int j = j0, tt = tt0;
#pragma unroll
      for (int v = 0; v < tpg; ++v) {
        off[v] = (t0 + v < a.Ktot) ? ((long)j * a.n_w) * a.n_ov + tt : -1;
        if (++tt == a.n_ov) {
          tt = 0;
          ++j;
        }
      }
    }
    unsigned long long xw[tpg];
#pragma unroll
    for (int v = 0; v < tpg; ++v) xw[v] = off[v] >= 0 ? __ldg(a.wx + off[v] + (long)a.w0 * a.n_ov) : 0ull;
    int eAw = a.eA[(long)a.w0 * a.Npad + P];
    for (int g = 0; g < a.G; ++g) {
      const int w = a.w0 + g;
      const int shbase = 30 + eAw - eC;
      // next frequency's weights and row exponent, in flight during this one
      unsigned long long xn[tpg];
      const bool more = g + 1 < a.G;
#pragma unroll
      for (int v = 0; v < tpg; ++v)
        xn[v] = (more && off[v] >= 0) ? __ldg(a.wx + off[v] + (long)(w + 1) * a.n_ov) : 0ull;
      const int eAn = more ? a.eA[(long)(w + 1) * a.Npad + P] : 0;
      uint32_t px[MAX_S][8];
      long long wm_prev = 0;
      int sh_prev = 0;
#pragma unroll
      for (int v = 0; v < tpg; ++v) {
        const unsigned long long x = xw[v];
        const long long wmv = (long long)(uint32_t)x;
        const int shv = shbase - (int)(uint32_t)(x >> 32);
        if constexpr (CPLX) {
          pair_x(round_shift(cv[2 * v], wmv, shv), round_shift(cv[2 * v + 1], wmv, shv), v, a.s, px);
        } else if ((v & 1) == 0) {
          wm_prev = wmv;
          sh_prev = shv;
        } else {
          pair_x(round_shift(cv[v - 1], wm_prev, sh_prev), round_shift(cv[v], wmv, shv), v >> 1, a.s, px);
        }
      }
      store_planes_x(a, g, P, tg, px);
#pragma unroll
      for (int v = 0; v < tpg; ++v) xw[v] = xn[v];
      eAw = eAn;
    }
  }
}

// ------------------------------------------- frequency-batched operand ----
// The transitions of a q are grouped into bins of their energy (positions u
// of a permuted K range, bin b holding [u0[b], u0[b+1]), padded to whole
// K-blocks); bin b's weighted operand is needed only for its own skeleton
// frequencies (slots).  One launch writes slots [g0, g0 + G[b]) of every
// bin: the digit planes of bin b go to S + aoff[b], blocked as
//   [slot g - g0][I = P/128][K-block of the bin][plane][4 KB core-matrix block],
// i.e. each bin is a weighted operand of its own over its K range.
constexpr int SB_MAX_BINS = 32;
struct SliceBinArgs {
  int cplx, Npad, Kr, s, n_kb, nb, g0, rmax, Kt;
  const int* cfix;               // [Npad][Kr], positions in bin order
  const int* eC;                 // [Npad] raw row maxima of the FP64 exponent field of C
  const unsigned long long* wx;  // [rmax][Kt] skeleton weights (mantissa | exponent << 32)
  const int* eAraw;              // [nb][rmax][Npad] raw row maxima of (exponent of c) + (exponent of w)
  uint16_t* S;
  int kb0[SB_MAX_BINS + 1];  // first K-block of each bin (kb0[nb] = n_kb)
  int G[SB_MAX_BINS];        // slots of each bin in this launch
  long aoff[SB_MAX_BINS];    // bin's plane offset in S (uint16 units)
};

template <bool CPLX>
__device__ __forceinline__ void slice_unit_bin(const SliceBinArgs& a, long idx) {
  constexpr int tpg = CPLX ? 8 : 16;  // positions per K-block
  const int P = (int)(idx % a.Npad);
  const int kb = (int)(idx / a.Npad);
  int b = 0;
  while (b + 1 < a.nb && a.kb0[b + 1] <= kb) ++b;
  const int G = a.G[b];
  if (G <= 0) return;
  const int kbl = kb - a.kb0[b];
  const long nkb = a.kb0[b + 1] - a.kb0[b];
  const long nI = a.Npad / 128;
  const int4* src = reinterpret_cast<const int4*>(a.cfix + (long)P * a.Kr + (long)kb * 16);
  int cv[16];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int4 x = src[v];
    cv[4 * v] = x.x;
    cv[4 * v + 1] = x.y;
    cv[4 * v + 2] = x.z;
    cv[4 * v + 3] = x.w;
  }
  const int rc = a.eC[P];
  const int eC = rc ? rc - 1022 : -2000;
  const long u0 = (long)kb * tpg;
  for (int gl = 0; gl < G; ++gl) {
    const int g = a.g0 + gl;
    const int ra = a.eAraw[((long)b * a.rmax + g) * a.Npad + P];
    const int eA = ra > 0 ? ra - 2044 + 1 : -2000;
    const int shbase = 30 + eA - eC;
    const unsigned long long* wr = a.wx + (long)g * a.Kt + u0;
    uint32_t px[MAX_S][8];
    long long wm_prev = 0;
    int sh_prev = 0;
#pragma unroll
    for (int v = 0; v < tpg; ++v) {
      const unsigned long long x = __ldg(wr + v);
      const long long wmv = (long long)(uint32_t)x;
      const int shv = shbase - (int)(uint32_t)(x >> 32);
      if constexpr (CPLX) {
        pair_x(round_shift(cv[2 * v], wmv, shv), round_shift(cv[2 * v + 1], wmv, shv), v, a.s, px);
      } else if ((v & 1) == 0) {
        wm_prev = wmv;
        sh_prev = shv;
      } else {
        pair_x(round_shift(cv[v - 1], wm_prev, sh_prev), round_shift(cv[v], wmv, shv), v >> 1, a.s, px);
      }
    }
#pragma unroll
    for (int i = 0; i < MAX_S; ++i) {
      if (i >= a.s) break;
      uint16_t* blk = a.S + a.aoff[b] + ((((long)gl * nI + (P >> 7)) * nkb + kbl) * a.s + i) * 2048;
      store_core_rows(blk, P & 127, px[i]);
    }
  }
}

}  // namespace
}  // namespace rpa
