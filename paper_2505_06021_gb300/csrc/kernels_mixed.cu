// Split-precision chi0 on the tcgen05 tensor cores of GB300 (sm_103a).
//
// chi0_PQ(q, w) = - sum_t conj(A_Pt) A_Qt with A = sqrt(zeta_k |d_t(w)|) C
// (the fit-basis response of Sec. 2.2; d_t < 0) is a dense Hermitian
// contraction over t = (k, i, a).  FP64 operands are turned into BF16 "digit
// slices" (Ozaki-style error-free splitting):
//
//   x = 2^(e_P - 7) * (v_0 + v_1 + v_2 + v_3),  v_i = d_i 2^(-8i),
//
// with one exponent e_P per row P, |d_0| <= 64 and |d_i| <= 128 integers (all
// exactly representable in BF16), obtained from the FP64 bit patterns with
// integer arithmetic only (GB300's FP64 pipe is 1/58 of FP32).  The products of
// slices (i, j) with i + j <= s - 1, plus (i, i) for 2i = s (it removes the
// systematic bias of the dropped level on the diagonal), are accumulated on the
// tensor cores in FP32 TMEM accumulators:
//   level 0  (d_0 d_0', integers): exact while |sum| <= 2^24, i.e. for 2048
//            complex t per flush;
//   level >= 1 (all other pairs, scaled by 2^-8 per level): FP32.
// Every 2048 t the accumulators are drained into float-float partial sums in
// global memory (L2-resident).  Complex data is kept planar (re, im planes);
//   Re += Ar Ar^T + Ai Ai^T,   Im += Ar Ai^T - Ai Ar^T
// use the instruction descriptor's negate-A bit for the minus sign.
// The K range of every output tile is split over several CTAs (split-K); a
// reduction kernel adds the float-float partials in a fixed order, applies the
// exponents and writes chi0 in FP64 (lower triangle + Hermitian mirror), so the
// result is deterministic.
//
// Tile: 128 rows (P) x 128 columns (Q) per CTA, K-blocks of 16 complex t;
// operands arrive by TMA (3-D tensor map over [plane][row][t], 32-byte
// swizzle), one elected thread issues tcgen05.mma, four epilogue warps drain
// TMEM with tcgen05.ld.  Every wait is bounded (globaltimer); on a time-out
// the kernel raises an error flag, drains its copies and frees TMEM.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "rpa_internal.h"

namespace rpa {
namespace {

constexpr int TILE = 128;          // rows and columns of an output tile
constexpr int KB = 16;             // complex t per K-block (= MMA K)
constexpr int CHUNK = 2048;        // t per exact level-0 accumulation
constexpr int KB_PER_CHUNK = CHUNK / KB;
constexpr int STAGES = 3;
constexpr int MAX_PLANES = 8;      // 4 slices x (re, im)
constexpr int PLANE_BYTES = TILE * KB * 2;  // 4096
constexpr int STAGE_BYTES = 2 * MAX_PLANES * PLANE_BYTES;  // A + B = 64 KB
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // producer, MMA, 4 epilogue warps
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per wait

// ------------------------------------------------------------ PTX helpers -

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and raises the flags) on time-out or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > WAIT_NS) {
      *abort_flag = 1;
      atomicCAS(err, 0, code);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (K-major, 32-byte swizzle): start >> 4,
// LBO = 16 B (unused for this layout), SBO = 256 B between 8-row groups,
// descriptor version 1, swizzle mode 6 (32 B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;
  return d;
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, K-major A and B,
// M = 128, N = 128, optional negation of A.
__device__ __forceinline__ uint32_t idesc(bool negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(TILE >> 3) << 17) |
         ((uint32_t)(TILE >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(a), "l"(b), "r"(id), "r"((uint32_t)acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// float-float helpers (Knuth TwoSum / Dekker FastTwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void ff_add(float& hi, float& lo, float a, float b) {
  // (hi, lo) += a + b, a and b floats
  float s, e, t, f;
  two_sum(a, b, s, e);
  two_sum(hi, s, t, f);
  f += lo + e;
  hi = t + f;
  lo = f - (hi - t);
}

// ------------------------------------------------------------ slicing -----
// x = c * w from the FP64 bit patterns: 30-bit rounded significands, 60-bit
// product, rounded to the fixed point F = round(x / 2^(e+1) * 2^32) with
// |F| < 2^30 whenever |x| < 2^(e-1).
__device__ __forceinline__ int fixed_point(double c, double w, int e) {
  const unsigned long long cb = (unsigned long long)__double_as_longlong(c);
  const unsigned long long wb = (unsigned long long)__double_as_longlong(w);
  const int Ec = (int)((cb >> 52) & 0x7ff), Ew = (int)((wb >> 52) & 0x7ff);
  if (Ec == 0 || Ew == 0) return 0;
  const unsigned long long mc = (((cb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) + (1ull << 22)) >> 23;  // <= 2^30
  const unsigned long long mw = (((wb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) + (1ull << 22)) >> 23;
  const unsigned long long p = mc * mw;  // <= 2^60
  const int sh = e + 2073 - Ec - Ew;  // >= 30 by the choice of e
  if (sh >= 62) return 0;
  if (sh < 30) return 0;  // unreachable when e bounds the row
  const int F = (int)((p + (1ull << (sh - 1))) >> sh);
  return (cb >> 63) ? -F : F;
}

__device__ __forceinline__ uint16_t bf16_of(int d, int lvl) {
  // d * 2^(-8 lvl) is exact in BF16 (|d| <= 128)
  const float f = (float)d * __int_as_float((127 - 8 * lvl) << 23);
  return (uint16_t)(__float_as_uint(f) >> 16);
}

struct SliceArgs {
  int cplx, N, Npad, n_ov, n_k, Ktot, Kpad, s, n_planes, n_w, w0, G;
  const double* const* C;  // [n_k] blocks of this q
  const double* wtab;      // [n_k][n_w][n_ov] sqrt(zeta |d|)
  const int* ecmax;        // [Npad] max exponent field of |C| per row
  const int* ewmax;        // [n_w] max exponent field of w per frequency
  uint16_t* S;             // [G][n_planes][Npad][Kpad]
  int* erow;               // [G][Npad] row exponents e_P
};

__global__ void __launch_bounds__(256) slice_kernel(SliceArgs a) {
  const long groups = (long)a.G * a.Npad * (a.Kpad / 8);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < groups; idx += (long)gridDim.x * blockDim.x) {
    long r = idx;
    const int tg = (int)(r % (a.Kpad / 8));
    r /= (a.Kpad / 8);
    const int P = (int)(r % a.Npad);
    const int g = (int)(r / a.Npad);
    const int w = a.w0 + g;
    const int e = (P < a.N) ? a.ecmax[P] + a.ewmax[w] - 2044 + 1 : 0;  // |x| < 2^(e-1)
    if (tg == 0) a.erow[(long)g * a.Npad + P] = e;
    uint32_t pk[MAX_PLANES][4];
#pragma unroll
    for (int pl = 0; pl < MAX_PLANES; ++pl)
#pragma unroll
      for (int u = 0; u < 4; ++u) pk[pl][u] = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int tglob = tg * 8 + u;
      int Fr = 0, Fi = 0;
      if (P < a.N && tglob < a.Ktot) {
        const int j = tglob / a.n_ov, t = tglob - j * a.n_ov;
        const double wv = a.wtab[((long)j * a.n_w + w) * a.n_ov + t];
        if (a.cplx) {
          const double2 cv = reinterpret_cast<const double2*>(a.C[j])[(long)P * a.n_ov + t];
          Fr = fixed_point(cv.x, wv, e);
          Fi = fixed_point(cv.y, wv, e);
        } else {
          Fr = fixed_point(a.C[j][(long)P * a.n_ov + t], wv, e);
        }
      }
      // signed digits: F = d0 2^24 + d1 2^16 + d2 2^8 + d3
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (c == 1 && !a.cplx) break;
        int F = c == 0 ? Fr : Fi;
        int d[4];
        d[0] = (F + (1 << 23)) >> 24;
        F -= d[0] << 24;
        d[1] = (F + (1 << 15)) >> 16;
        F -= d[1] << 16;
        d[2] = (F + (1 << 7)) >> 8;
        F -= d[2] << 8;
        d[3] = F;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (i >= a.s) break;
          const int pl = a.cplx ? 2 * i + c : i;
          const uint32_t h = bf16_of(d[i], i);
          pk[pl][u >> 1] |= (u & 1) ? (h << 16) : h;
        }
      }
    }
    for (int pl = 0; pl < a.n_planes; ++pl) {
      uint4* dst = reinterpret_cast<uint4*>(a.S + (((long)g * a.n_planes + pl) * a.Npad + P) * a.Kpad + tg * 8);
      *dst = make_uint4(pk[pl][0], pk[pl][1], pk[pl][2], pk[pl][3]);
    }
  }
}

// max exponent field of |C| over all t of row P (all k-pairs of this q)
__global__ void __launch_bounds__(256) cexp_kernel(int cplx, int N, int n_ov, int n_k, const double* const* C,
                                                   int* ecmax) {
  const int P = blockIdx.x;
  int m = 0;
  const long per = (long)n_ov * (cplx ? 2 : 1);
  for (int j = 0; j < n_k; ++j) {
    const unsigned long long* row =
        reinterpret_cast<const unsigned long long*>(C[j]) + (long)P * per;
    for (long t = threadIdx.x; t < per; t += blockDim.x) m = max(m, (int)((row[t] >> 52) & 0x7ff));
  }
  __shared__ int red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) ecmax[P] = red[0];
}

// w = sqrt(zeta_k |d|) and the max exponent field of w per frequency
__global__ void __launch_bounds__(256) wtab_kernel(int n_k, int n_w, int n_ov, const double* dtab, double* wtab,
                                                   int* ewmax) {
  const int w = blockIdx.x;
  int m = 0;
  for (int j = 0; j < n_k; ++j)
    for (int t = threadIdx.x; t < n_ov; t += blockDim.x) {
      const long i = ((long)j * n_w + w) * n_ov + t;
      const double v = sqrt(fabs(dtab[i]));
      wtab[i] = v;
      m = max(m, (int)((__double_as_longlong(v) >> 52) & 0x7ff));
    }
  __shared__ int red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) ewmax[w] = red[0];
}

// ---------------------------------------------------------- GEMM kernel ----

struct TcArgs {
  int cplx, s, n_planes;
  int n_tiles, n_ksplit, chunks_per_split, n_chunks;
  int n_items;
  float* part;  // [item][4][TILE cols][TILE rows]: Re_hi, Re_lo, Im_hi, Im_lo
  int* err;
  int pair_i[16], pair_j[16], pair_lvl[16], n_pairs;
};

__device__ __forceinline__ void tri_idx(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// item -> (g, tile, ksplit)
__device__ __forceinline__ void item_coords(const TcArgs& a, int item, int& g, int& I, int& J, int& ks) {
  ks = item % a.n_ksplit;
  int r = item / a.n_ksplit;
  const int tile = r % a.n_tiles;
  g = r / a.n_tiles;
  tri_idx(tile, I, J);
}

__global__ void __launch_bounds__(THREADS, 1) chi0_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 32 * EPI_WARPS);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int plane_bytes_total = a.n_planes * PLANE_BYTES;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[STAGES];
      for (int i = 0; i < STAGES; ++i) armed[i] = -1;
      bool ok = true;
      for (int item = blockIdx.x; item < a.n_items && ok; item += gridDim.x) {
        int g, I, J, ks;
        item_coords(a, item, g, I, J, ks);
        const int c0 = ks * a.chunks_per_split, c1 = min(a.n_chunks, c0 + a.chunks_per_split);
        for (int kb = c0 * KB_PER_CHUNK; kb < c1 * KB_PER_CHUNK && ok; ++kb) {
          ok = mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err, 11);
          if (!ok) break;
          uint8_t* sa = smem + stage * STAGE_BYTES;
          uint8_t* sb = sa + MAX_PLANES * PLANE_BYTES;
          mbar_expect_tx(&full[stage], 2 * plane_bytes_total);
          tma_load_3d(sa, &tmap, &full[stage], kb * KB, I * TILE, g * a.n_planes);
          tma_load_3d(sb, &tmap, &full[stage], kb * KB, J * TILE, g * a.n_planes);
          armed[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // drain: every armed stage's copy must have landed before the CTA exits
      for (int i = 0; i < STAGES; ++i) {
        if (armed[i] < 0) continue;
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[i], (uint32_t)armed[i]) && gtime() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool ok = true;
      const uint32_t id_pos = idesc(false), id_neg = idesc(true);
      for (int item = blockIdx.x; item < a.n_items && ok; item += gridDim.x) {
        int g, I, J, ks;
        item_coords(a, item, g, I, J, ks);
        const int c0 = ks * a.chunks_per_split, c1 = min(a.n_chunks, c0 + a.chunks_per_split);
        for (int ch = c0; ch < c1 && ok; ++ch) {
          ok = mbar_wait(acc_empty, acc_phase ^ 1u, abort_flag, a.err, 12);
          if (!ok) break;
          fence_after();
          for (int kk = 0; kk < KB_PER_CHUNK && ok; ++kk) {
            ok = mbar_wait(&full[stage], phase, abort_flag, a.err, 13);
            if (!ok) break;
            fence_after();
            const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t sb = sa + MAX_PLANES * PLANE_BYTES;
            bool init0 = kk == 0, init1 = kk == 0;  // first MMA into each level this chunk
            for (int pi = 0; pi < a.n_pairs; ++pi) {
              const int i = a.pair_i[pi], j = a.pair_j[pi], lvl = a.pair_lvl[pi];
              const uint32_t dre = tmem + (lvl ? 256u : 0u), dim = dre + 128u;
              bool& first = lvl ? init1 : init0;
              if (a.cplx) {
                const uint64_t ar = sdesc(sa + (2 * i) * PLANE_BYTES), ai = sdesc(sa + (2 * i + 1) * PLANE_BYTES);
                const uint64_t br = sdesc(sb + (2 * j) * PLANE_BYTES), bi = sdesc(sb + (2 * j + 1) * PLANE_BYTES);
                mma(dre, ar, br, id_pos, !first);
                mma(dim, ar, bi, id_pos, !first);
                mma(dre, ai, bi, id_pos, true);
                mma(dim, ai, br, id_neg, true);
              } else {
                const uint64_t ar = sdesc(sa + i * PLANE_BYTES), br = sdesc(sb + j * PLANE_BYTES);
                mma(dre, ar, br, id_pos, !first);
              }
              first = false;
            }
            mma_commit(&empty[stage]);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (ok) mma_commit(acc_full);
          acc_phase ^= 1u;
        }
      }
      // all MMAs issued by this thread must be complete before TMEM is freed
      mma_commit(drain);
      const unsigned long long t0 = gtime();
      while (!mbar_try(drain, 0) && gtime() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ------------------------------------------------ epilogue (4 warps)
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < a.n_items && ok; item += gridDim.x) {
      int g, I, J, ks;
      item_coords(a, item, g, I, J, ks);
      const int c0 = ks * a.chunks_per_split, c1 = min(a.n_chunks, c0 + a.chunks_per_split);
      float* part = a.part + (long)item * 4 * TILE * TILE;
      for (int ch = c0; ch < c1 && ok; ++ch) {
        ok = mbar_wait(acc_full, acc_phase, abort_flag, a.err, 14);
        if (!ok) break;
        fence_after();
        const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
        const int n_parts = a.cplx ? 2 : 1;
        for (int c = 0; c < TILE; c += 16) {
          for (int part_k = 0; part_k < n_parts; ++part_k) {  // 0 = Re, 1 = Im
            float v0[16], v1[16];
            tmem_ld16(tl + part_k * 128 + c, v0);
            tmem_ld16(tl + 256 + part_k * 128 + c, v1);
            tmem_wait_ld();
            float* ph = part + ((long)(2 * part_k) * TILE) * TILE;
            float* pl = ph + (long)TILE * TILE;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const long o = (long)(c + u) * TILE + row;
              float hi = 0.f, lo = 0.f;
              if (ch != c0) {
                hi = ph[o];
                lo = pl[o];
              }
              ff_add(hi, lo, v0[u], v1[u]);
              ph[o] = hi;
              pl[o] = lo;
            }
          }
        }
        fence_before();
        mbar_arrive(acc_empty);
        acc_phase ^= 1u;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Sum of the split-K partials in a fixed order, exponents, Hermitian store.
struct ReduceArgs {
  int cplx, N, Npad, n_tiles, n_ksplit, w0, G;
  const float* part;
  const int* erow;  // [G][Npad]
  double* chi;      // [n_w][N][N] of this q
};

__global__ void __launch_bounds__(256) reduce_kernel(ReduceArgs a) {
  const int tile = blockIdx.x % a.n_tiles;
  const int g = blockIdx.x / a.n_tiles;
  int I, J;
  tri_idx(tile, I, J);
  const long NN = (long)a.N * a.N;
  double* out = a.chi + (long)(a.w0 + g) * NN * (a.cplx ? 2 : 1);
  for (int idx = threadIdx.x; idx < TILE * TILE; idx += blockDim.x) {
    const int c = idx / TILE, r = idx % TILE;  // part layout [col][row]
    const int P = I * TILE + r, Q = J * TILE + c;
    if (P >= a.N || Q >= a.N || Q > P) continue;
    double re = 0.0, im = 0.0;
    for (int ks = 0; ks < a.n_ksplit; ++ks) {
      const long item = ((long)g * a.n_tiles + tile) * a.n_ksplit + ks;
      const float* p = a.part + item * 4 * TILE * TILE + idx;
      re += (double)p[0] + (double)p[TILE * TILE];
      if (a.cplx) im += (double)p[2 * TILE * TILE] + (double)p[3 * TILE * TILE];
    }
    const int e = a.erow[(long)g * a.Npad + P] + a.erow[(long)g * a.Npad + Q];
    const double sc = -ldexp(1.0, e - 14);  // x = 2^(e_P - 7) * sum v, chi = -sum conj(x) x
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

struct MixedLayout {
  int Npad, Kpad, Ktot, n_planes, G, n_tiles, n_ksplit, chunks_per_split, n_chunks, n_items;
  size_t slices, erow, part, ecmax, ewmax, wtab, err, total;
};

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

MixedLayout mixed_layout(const BatchGeom& g, int s, int sms) {
  MixedLayout L{};
  L.Npad = (g.n_aux + TILE - 1) / TILE * TILE;
  L.Ktot = g.n_k * g.n_ov;
  L.Kpad = (L.Ktot + CHUNK - 1) / CHUNK * CHUNK;
  L.n_planes = g.cplx ? 2 * s : s;
  L.n_chunks = L.Kpad / CHUNK;
  const int nb = L.Npad / TILE;
  L.n_tiles = nb * (nb + 1) / 2;
  const size_t per_w = (size_t)L.n_planes * L.Npad * L.Kpad * 2;
  // frequencies per launch: slices of at most ~12 GB
  L.G = (int)std::max<size_t>(1, std::min<size_t>(g.n_w, ((size_t)12 << 30) / per_w));
  // split K so that a launch has about four items per SM
  const int want = 4 * sms;
  L.n_ksplit = std::max(1, std::min(L.n_chunks, (want + L.G * L.n_tiles - 1) / (L.G * L.n_tiles)));
  L.chunks_per_split = (L.n_chunks + L.n_ksplit - 1) / L.n_ksplit;
  L.n_ksplit = (L.n_chunks + L.chunks_per_split - 1) / L.chunks_per_split;
  L.n_items = L.G * L.n_tiles * L.n_ksplit;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  L.slices = al(per_w * L.G);
  L.erow = al(sizeof(int) * L.G * L.Npad);
  L.part = al(sizeof(float) * 4 * TILE * TILE * (size_t)L.n_items);
  L.ecmax = al(sizeof(int) * L.Npad);
  L.ewmax = al(sizeof(int) * g.n_w);
  L.wtab = al(sizeof(double) * (size_t)g.n_k * g.n_w * g.n_ov);
  L.err = al(sizeof(int) * 4);
  L.total = L.slices + L.erow + L.part + L.ecmax + L.ewmax + L.wtab + L.err;
  return L;
}

}  // namespace

bool mixed_supported() { return get_encode() != nullptr; }

size_t mixed_workspace_bytes(const BatchGeom& g, int n_slices) { return mixed_layout(g, n_slices, num_sms()).total; }

cudaError_t launch_chi0_mixed(const BatchGeom& g, int s, const double* const* Cptrs, const double* dtab,
                              double* chi, void* work, size_t work_bytes, int* status, uint64_t* n_launch,
                              cudaStream_t st) {
  if (s < 2 || s > 4) return cudaErrorInvalidValue;
  EncodeTiledFn enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  const int sms = num_sms();
  MixedLayout L = mixed_layout(g, s, sms);
  if (L.total > work_bytes) return cudaErrorMemoryAllocation;
  char* p = (char*)work;
  uint16_t* S = (uint16_t*)p;
  p += L.slices;
  int* erow = (int*)p;
  p += L.erow;
  float* part = (float*)p;
  p += L.part;
  int* ecmax = (int*)p;
  p += L.ecmax;
  int* ewmax = (int*)p;
  p += L.ewmax;
  double* wtab = (double*)p;
  p += L.wtab;
  int* err = (int*)p;

  static thread_local int attr_done = 0;
  const size_t smem = STAGES * STAGE_BYTES + 1024 + 256;  // stages, alignment pad, barriers
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(chi0_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = 1;
  }
  uint64_t nl = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return e;
  cexp_kernel<<<g.n_aux, 256, 0, st>>>(g.cplx, g.n_aux, g.n_ov, g.n_k, Cptrs, ecmax);
  wtab_kernel<<<g.n_w, 256, 0, st>>>(g.n_k, g.n_w, g.n_ov, dtab, wtab, ewmax);
  nl += 2;
  // tensor map over the slice buffer: dims (t: Kpad, row: Npad, plane: G*n_planes)
  CUtensorMap tmap;
  cuuint64_t dims[3] = {(cuuint64_t)L.Kpad, (cuuint64_t)L.Npad, (cuuint64_t)L.G * L.n_planes};
  cuuint64_t strides[2] = {(cuuint64_t)L.Kpad * 2, (cuuint64_t)L.Kpad * 2 * L.Npad};
  cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)TILE, (cuuint32_t)L.n_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, S, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TcArgs ta{};
  ta.cplx = g.cplx;
  ta.s = s;
  ta.n_planes = L.n_planes;
  ta.n_tiles = L.n_tiles;
  ta.n_ksplit = L.n_ksplit;
  ta.chunks_per_split = L.chunks_per_split;
  ta.n_chunks = L.n_chunks;
  ta.part = part;
  ta.err = err;
  int np = 0;
  for (int lvl = 0; lvl < s; ++lvl)
    for (int i = 0; i <= lvl; ++i) {
      ta.pair_i[np] = i;
      ta.pair_j[np] = lvl - i;
      ta.pair_lvl[np] = lvl ? 1 : 0;
      ++np;
    }
  if (s % 2 == 0) {  // (s/2, s/2): removes the diagonal bias of the dropped level
    ta.pair_i[np] = s / 2;
    ta.pair_j[np] = s / 2;
    ta.pair_lvl[np] = 1;
    ++np;
  }
  ta.n_pairs = np;
  for (int w0 = 0; w0 < g.n_w; w0 += L.G) {
    const int G = std::min(L.G, g.n_w - w0);
    SliceArgs sa{g.cplx, g.n_aux, L.Npad, g.n_ov, g.n_k, L.Ktot, L.Kpad, s, L.n_planes, g.n_w, w0, G,
                 Cptrs, wtab, ecmax, ewmax, S, erow};
    const long groups = (long)G * L.Npad * (L.Kpad / 8);
    const long blocks = std::min<long>((groups + 255) / 256, (long)sms * 32);
    slice_kernel<<<(unsigned)blocks, 256, 0, st>>>(sa);
    ta.n_items = G * L.n_tiles * L.n_ksplit;
    const int grid = std::min(ta.n_items, sms);
    chi0_tc_kernel<<<grid, THREADS, smem, st>>>(tmap, ta);
    ReduceArgs ra{g.cplx, g.n_aux, L.Npad, L.n_tiles, L.n_ksplit, w0, G, part, erow, chi};
    reduce_kernel<<<G * L.n_tiles, 256, 0, st>>>(ra);
    nl += 3;
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

}  // namespace rpa
