// The tensor-core kernel of the split-precision chi0 (GB300, sm_103a):
// constants, PTX helpers (mbarrier, bulk copy, tcgen05) and chi0_tc_kernel.
// Included once, by kernels_mixed.cu, which holds the operand preparation,
// the split-K reduction and the host launcher.
//
// Tile: 128 rows P x 64 complex columns Q (128 x 128 for real data), K-blocks
// of 16 real values; operands arrive by bulk copies of pre-blocked digit
// planes (one contiguous 16 KB run per operand and K-block, no-swizzle
// core-matrix layout), one elected thread issues tcgen05.mma, eight epilogue
// warps drain TMEM with tcgen05.ld, and two slicer warps may write another
// q's weighted digit planes meanwhile (a side job without waits).  Slice pairs are grouped by level into
// four TMEM accumulators (levels 0-2 exact, levels >= 3 FP32); every CHUNK t
// the epilogue adds them into float-float register accumulators.  Every wait
// is bounded (globaltimer); on a time-out the kernel raises an error flag,
// lets its copies land, waits for its MMAs and frees TMEM.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "slice.cuh"

namespace rpa {
namespace {

constexpr int KB = 16;              // real K per K-block (= MMA K for BF16)
constexpr int CHUNK = 1024;         // complex t per exact accumulation (real: 2048 t)
constexpr int STAGES = 6;
constexpr int PLANE_BYTES = 128 * KB * 2;                 // 4096: one slice, 128 rows, 16 values
constexpr int STAGE_BYTES = 2 * MAX_S * PLANE_BYTES;      // A + B = 32 KB
constexpr int EPI_WARPS = 8;
constexpr int SLICE_WARPS = 2;
constexpr int THREADS = 64 + 32 * EPI_WARPS + 32 * SLICE_WARPS;  // producer, MMA, epilogue, slicer warps
constexpr int NGROUPS = 4;
constexpr unsigned long long WAIT_NS = 2000000000ull;     // 2 s per wait

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
// try_wait with a suspend-time hint: a waiting thread sleeps until the phase
// completes or about `ns` nanoseconds pass, instead of spinning on the barrier
// and stealing issue slots from the producer and MMA threads.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and raises the flags) on time-out or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code, uint32_t sleep_ns = 0) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (sleep_ns ? mbar_try_sleep(b, parity, sleep_ns) : mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > WAIT_NS) {
      *abort_flag = 1;
      atomicCAS(err, 0, code);
      return false;
    }
  }
}
// Contiguous global -> shared copy completing on an mbarrier (addresses 16-byte
// aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major without swizzle: start >> 4,
// LBO = 128 B between K-adjacent core matrices, SBO = 256 B between 8-row
// groups, descriptor version 1, swizzle mode 0.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, K-major A and B,
// M = 128, N = 128 or 256.
__device__ __forceinline__ uint32_t idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// float-float accumulation (Knuth TwoSum, Dekker FastTwoSum):
// (hi, lo) += g0 + g1 + g2 + g3, with g0, g1 integer-valued and exact, g2, g3
// small (their FP32 sum is accurate to 2^-24 of a 2^-16-level quantity).
__device__ __forceinline__ void ff_add4(float& hi, float& lo, float g0, float g1, float g2, float g3) {
  float s = g0 + g1;
  float bb = s - g0;
  float e = (g0 - (s - bb)) + (g1 - bb);
  e += g2 + g3;
  float t = hi + s;
  float b2 = t - hi;
  float f = (hi - (t - b2)) + (s - b2);
  f += lo + e;
  hi = t + f;
  lo = f - (hi - t);
}

// ---------------------------------------------------------- GEMM kernel ----
// One persistent launch covers several "segments": a segment is one q of one
// job with G frequencies, its own operand buffers and partial buffer.  The
// segment table travels in the kernel parameters, so a launch needs no
// device-side table and records cleanly into a CUDA graph.  Operand data
// arrives by plain bulk copies (cp.async.bulk): the digit planes are stored
// pre-blocked, one contiguous 16 KB run per operand and K-block.

constexpr int MAX_SEGS = 96;

struct TcSeg {
  const uint16_t* A;  // weighted digit planes, [g][I][kb][plane][4 KB block]
  const uint16_t* B;  // digit planes of C, [J][ldb][plane][4 KB block]; this segment reads K-blocks kb_off + kb
  float* part;        // [item][2 (hi, lo)][128 rows][128 cols]
  int cplx, G, n_tiles, n_ksplit, kb_per_split, n_kb, item0, nI;
  int kb_off, ldb;    // the segment's K range within B, B's K-blocks per column block
};

struct TcParams {
  int n_segs, n_items, s, kb_per_chunk;
  int drop_item;  // test hook: the first K-block of this work item is never
                  // loaded (-1: off), so one bounded wait runs out
  int* err;
  int grp_mask;  // accumulator groups that receive MMAs (the host's copy of MmaTable<s>::mask)
  // Side job of the slicer warps: the weighted digit planes of another q
  // (all its frequencies), written while this launch's MMAs run; its inputs
  // and output share nothing with this launch's segments.
  int side_on;        // 1: side (per-frequency operand), 2: sideb (frequency-batched operand)
  SliceArgs side;
  SliceBinArgs sideb;
  TcSeg seg[MAX_SEGS];
};
static_assert(sizeof(TcParams) <= 32000, "kernel parameter block too large");

// complex: row blocks of 128, column blocks of 64, tiles with J <= 2I + 1;
// real: 128 x 128 lower tiles
__device__ __forceinline__ void tile_ij(int cplx, int t, int& I, int& J) {
  if (cplx) {
    int i = (int)((sqrtf(4.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) <= t) ++i;
    while (i * (i + 1) > t) --i;
    I = i;
    J = t - i * (i + 1);
  } else {
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    I = i;
    J = t - i * (i + 1) / 2;
  }
}

struct ItemPos {
  int seg, local, g, I, J, ks, kb0, kb1;
};

// Within a segment: local = (ks * G + g) * n_tiles + tile.  CTAs that run at
// the same time work on the same K range, so the frequency-independent B
// operand (slices of C) and the A rows are read from HBM about once and shared
// in L2.
__device__ __forceinline__ ItemPos item_pos(const TcParams& p, int item) {
  ItemPos r;
  int sg = 0;
  while (sg + 1 < p.n_segs && p.seg[sg + 1].item0 <= item) ++sg;
  const TcSeg& S = p.seg[sg];
  r.seg = sg;
  r.local = item - S.item0;
  const int tile = r.local % S.n_tiles;
  const int q = r.local / S.n_tiles;
  r.g = q % S.G;
  r.ks = q / S.G;
  tile_ij(S.cplx, tile, r.I, r.J);
  r.kb0 = r.ks * S.kb_per_split;
  r.kb1 = min(S.n_kb, r.kb0 + S.kb_per_split);
  return r;
}

// The MMAs of one K-block.  Slice pairs (i, j) of S digit planes: all levels
// i + j < S, and for S = 2 also (1, 1) (the largest term of level 2);
// accumulator group = min(level, 3), TMEM columns [128 g, 128 g + 128).  For S
// = 4 the dropped level-4 terms are 2^-32 of level 0 (measured |dE_c| 2.9e-9 Ha
// on the 2-D periodic job).  Two pairs (i, j), (i, j + 1) whose groups are g,
// g + 1 with g even share one MMA of N = 256: B's digit planes j and j + 1 are
// adjacent in the stage (4 KB apart, the 8-row-group stride continuing), so
// they form one 256-row operand, and the two groups one 256-column TMEM range
// at a 256-aligned offset; the A tile is read from shared memory once for both.
// `first` marks an MMA whose groups receive nothing earlier in the stage (it
// starts their sums at the first K-block of a chunk); pairs are merged only
// where that holds for both groups or for neither.  S = 4: 6 MMAs (4 wide)
// for the 10 pairs; S = 3: 5 for 6; S = 2: 3 for 4.
template <int S>
struct MmaTable {
  int n, i[16], j[16], g[16], wide[16], first[16], mask;
  static constexpr int grp(int level) { return level < NGROUPS - 1 ? level : NGROUPS - 1; }
  static constexpr bool in(int a, int b) { return a < S && b < S && (a + b < S || (S == 2 && a == 1 && b == 1)); }
  constexpr MmaTable() : n(0), i(), j(), g(), wide(), first(), mask(0) {
    bool touched[NGROUPS] = {};
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S;) {
        if (!in(a, b)) {
          ++b;
          continue;
        }
        const int g0 = grp(a + b);
        const bool w = in(a, b + 1) && g0 % 2 == 0 && grp(a + b + 1) == g0 + 1 && touched[g0] == touched[g0 + 1];
        i[n] = a;
        j[n] = b;
        g[n] = g0;
        wide[n] = w;
        first[n] = !touched[g0];
        touched[g0] = true;
        mask |= 1 << g0;
        if (w) {
          touched[g0 + 1] = true;
          mask |= 1 << (g0 + 1);
        }
        ++n;
        b += w ? 2 : 1;
      }
  }
};

// Compile-time check of the table: every pair of the set lands in exactly one
// MMA, in the group of its level, and `first` is set exactly on the first MMA
// into each of its groups.
template <int S>
constexpr bool mma_table_ok() {
  constexpr MmaTable<S> t{};
  using T = MmaTable<S>;
  for (int a = 0; a < MAX_S; ++a)
    for (int b = 0; b < MAX_S; ++b) {
      int c = 0;
      for (int m = 0; m < t.n; ++m)
        if (t.i[m] == a && (t.j[m] == b || (t.wide[m] && t.j[m] + 1 == b))) {
          ++c;
          if (T::grp(a + b) != t.g[m] + b - t.j[m]) return false;
        }
      if (c != (T::in(a, b) ? 1 : 0)) return false;
    }
  for (int m = 0; m < t.n; ++m)
    for (int h = 0; h <= t.wide[m]; ++h) {
      bool earlier = false;
      for (int k = 0; k < m; ++k)
        if (t.g[k] == t.g[m] + h || (t.wide[k] && t.g[k] + 1 == t.g[m] + h)) earlier = true;
      if (earlier == (t.first[m] != 0)) return false;
    }
  return true;
}
static_assert(mma_table_ok<2>() && mma_table_ok<3>() && mma_table_ok<4>(), "slice-pair MMA table is inconsistent");
static_assert(MmaTable<4>{}.n == 6 && MmaTable<3>{}.n == 5 && MmaTable<2>{}.n == 3, "unexpected MMA counts");

template <int S>
__device__ constexpr MmaTable<S> kMmas{};

template <int S>
__global__ void __launch_bounds__(THREADS, 1) chi0_tc_kernel(const __grid_constant__ TcParams p) {
  constexpr const MmaTable<S>& MT = kMmas<S>;
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
  constexpr uint32_t stage_tx = 2u * (uint32_t)S * PLANE_BYTES;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed[STAGES];
      for (int i = 0; i < STAGES; ++i) armed[i] = -1;
      bool ok = true;
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const ItemPos it = item_pos(p, item);
        const TcSeg& SG = p.seg[it.seg];
        for (int kb = it.kb0; kb < it.kb1 && ok; ++kb) {
          ok = mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.err, 11, 2000);
          if (!ok) break;
          uint8_t* sa = smem + stage * STAGE_BYTES;
          uint8_t* sb = sa + MAX_S * PLANE_BYTES;
          if (item == p.drop_item && kb == it.kb0) {  // nothing more issued: the MMA thread's wait runs out
            ok = false;
            break;
          }
          mbar_expect_tx(&full[stage], stage_tx);
          // A: X slices of rows I*128.. ; B: [X; Y] slices of columns J*64.. (real: X of J*128..)
          bulk_load(sa, SG.A + (((size_t)it.g * SG.nI + it.I) * SG.n_kb + kb) * (S * 2048), S * PLANE_BYTES,
                    &full[stage]);
          bulk_load(sb, SG.B + ((size_t)it.J * SG.ldb + SG.kb_off + kb) * (S * 2048), S * PLANE_BYTES,
                    &full[stage]);
          armed[stage] = (int)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // every armed stage's copy must have landed before the CTA exits
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
      const uint32_t id128 = idesc(128), id256 = idesc(256);
      // descriptors: plane 0 of stage 0, advanced by byte offsets >> 4
      const uint64_t d0 = sdesc(smem_u32(smem));
      for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const ItemPos it = item_pos(p, item);
        for (int c0 = it.kb0; c0 < it.kb1 && ok; c0 += p.kb_per_chunk) {
          const int c1 = min(it.kb1, c0 + p.kb_per_chunk);
          ok = mbar_wait(acc_empty, acc_phase ^ 1u, abort_flag, p.err, 12);
          if (!ok) break;
          fence_after();
          for (int kb = c0; kb < c1 && ok; ++kb) {
            ok = mbar_wait(&full[stage], phase, abort_flag, p.err, 13);
            if (!ok) break;
            fence_after();
            const uint64_t da = d0 + (uint64_t)((stage * STAGE_BYTES) >> 4);
            const uint64_t db = da + (uint64_t)((MAX_S * PLANE_BYTES) >> 4);
            const bool first_kb = kb == c0;
#pragma unroll
            for (int m = 0; m < MT.n; ++m)
              mma(tmem + 128u * (uint32_t)MT.g[m], da + (uint64_t)((MT.i[m] * PLANE_BYTES) >> 4),
                  db + (uint64_t)((MT.j[m] * PLANE_BYTES) >> 4), MT.wide[m] ? id256 : id128,
                  !(first_kb && MT.first[m]));
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
  } else if (warp < 2 + EPI_WARPS) {
    // ------------------------------------------------ epilogue (8 warps)
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // columns [64 half, 64 half + 64)
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(64 * half);
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
      const ItemPos it = item_pos(p, item);
      float hi[64], lo[64];
#pragma unroll
      for (int u = 0; u < 64; ++u) hi[u] = lo[u] = 0.f;
      for (int c0 = it.kb0; c0 < it.kb1 && ok; c0 += p.kb_per_chunk) {
        ok = mbar_wait(acc_full, acc_phase, abort_flag, p.err, 14, 20000);
        if (!ok) break;
        fence_after();
#pragma unroll
        for (int c = 0; c < 64; c += 8) {
          float v0[8], v1[8], v2[8], v3[8];
          tmem_ld8(tl + c, v0);
          tmem_ld8(tl + 128 + c, v1);
          if (p.grp_mask & 4) tmem_ld8(tl + 256 + c, v2);
          if (p.grp_mask & 8) tmem_ld8(tl + 384 + c, v3);
          tmem_wait_ld();
          if (!(p.grp_mask & 4))
#pragma unroll
            for (int u = 0; u < 8; ++u) v2[u] = 0.f;
          if (!(p.grp_mask & 8))
#pragma unroll
            for (int u = 0; u < 8; ++u) v3[u] = 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u) ff_add4(hi[c + u], lo[c + u], v0[u], v1[u], v2[u], v3[u]);
        }
        fence_before();
        mbar_arrive(acc_empty);
        acc_phase ^= 1u;
      }
      if (!ok) break;
      float* ph = p.seg[it.seg].part + (long)it.local * 2 * 128 * 128 + (long)row * 128 + 64 * half;
      float* pl = ph + 128 * 128;
#pragma unroll
      for (int u = 0; u < 64; u += 4) {
        *reinterpret_cast<float4*>(ph + u) = make_float4(hi[u], hi[u + 1], hi[u + 2], hi[u + 3]);
        *reinterpret_cast<float4*>(pl + u) = make_float4(lo[u], lo[u + 1], lo[u + 2], lo[u + 3]);
      }
    }
  } else if (p.side_on == 1) {
    // ------------------------------------------------ slicer (2 warps)
    // no waits: independent loads and stores, consecutive threads on
    // consecutive rows of one K-block as in the standalone slicing kernel
    constexpr int NT = 32 * SLICE_WARPS;
    const long total = (long)p.side.Npad * (p.side.Kr / 16);
    const long stride = (long)gridDim.x * NT;
    const long first = (long)blockIdx.x * NT + (threadIdx.x - (THREADS - NT));
    if (p.side.cplx) {
      for (long idx = first; idx < total; idx += stride) slice_unit<true, true>(p.side, idx);
    } else {
      for (long idx = first; idx < total; idx += stride) slice_unit<false, true>(p.side, idx);
    }
  } else if (p.side_on == 2) {
    // the same for the frequency-batched operand of another q
    constexpr int NT = 32 * SLICE_WARPS;
    const long total = (long)p.sideb.Npad * p.sideb.n_kb;
    const long stride = (long)gridDim.x * NT;
    const long first = (long)blockIdx.x * NT + (threadIdx.x - (THREADS - NT));
    if (p.sideb.cplx) {
      for (long idx = first; idx < total; idx += stride) slice_unit_bin<true>(p.sideb, idx);
    } else {
      for (long idx = first; idx < total; idx += stride) slice_unit_bin<false>(p.sideb, idx);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

}  // namespace
}  // namespace rpa
