// Exact clutter-resistant search on the tcgen05 tensor cores (sm_103a).
//
// Listing 1's distance splits into a needle constant and two cross terms:
//   d(i,j) = sum_k m_ik (a_ik - b_jk)^2 = A_i + S_ij,
//   A_i = sum_k a_ik^2,   S_ij = sum_k m_ik b_jk^2 - 2 a_ik b_jk,
// with a, b the column deltas (delta of column 0 := 0) and m_ik = [a_ik != 0] (m a = a).
// S is one GEMM with K = 2 N^2:  needle row [m_i | a_i]  x  haystack row [b_j^2 | -2 b_j].
//
// Exactness (the fp16 class): a needle is in the class when every |a| <= 127, a haystack image
// when every |b| <= 45 and S2_j + 254 S1_j < 2^24, with S2_j = sum_k b_jk^2 and
// S1_j = sum_k |b_jk|.  Every operand is then an integer exactly representable in fp16 (m, a;
// b^2 <= 2025 < 2^11, |2b| <= 90), every product is an exact integer, and every partial sum of
// any subset of the products m_ik b_jk^2 - 2 a_ik b_jk is an integer of magnitude at most
// S2_j + 2 * 127 * S1_j < 2^24, so the FP32 accumulation in TMEM is exact in any order.  Pairs
// with a side outside the class go to the CUDA-core kernels (dense int8 or exact int64).  The rank test S_ij < d(i,match_i) - A_i, and the top-1 key
// (A_i + S_ij, j), are evaluated in the GEMM epilogue; S is never written to memory.
//
// Kernel structure (one CTA per SM, persistent over 128 x 256 output tiles):
//   warp 0: TMA producer (128B-swizzled K-major tiles, 4-stage mbarrier pipeline)
//   warp 1: TMEM allocator and single-thread tcgen05.mma issuer (M=128, N=256, K=16)
//   warps 2-5: epilogue; tcgen05.ld of the accumulator (double-buffered: 2 x 256 columns)
// Every wait on an mbarrier gives up after 2 s of %globaltimer, sets RICI_ERR_TIMEOUT and lets
// the CTA reach its teardown (TMEM is always freed).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rici {
namespace {

constexpr int kBM = 128;          // needles per tile (TMEM lanes)
constexpr int kBN = 256;          // haystack images per tile (TMEM columns per buffer)
constexpr int kBK = 64;           // fp16 elements per k-block (one 128-byte swizzle row)
constexpr int kStages = 4;
constexpr int kTcThreads = 192;   // 6 warps
constexpr uint32_t kStageA = kBM * kBK * 2;  // 16 KB
constexpr uint32_t kStageB = kBN * kBK * 2;  // 32 KB
constexpr int kNarrowA = 127;     // |delta| limit of fp16-class needles (int8)
constexpr int kNarrowB = 45;      // |delta| limit of fp16-class haystack images (b^2 < 2^11)
constexpr int64_t kExactSum = 1ll << 24;  // bound on every partial sum (exact FP32 integers)
constexpr unsigned long long kNoBestTc = ~0ull;
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;
constexpr unsigned long long kDrainBudgetNs = 200000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false (and RICI_ERR_TIMEOUT) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status,
                                          int *abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int *)abort_flag) return false;
    if (globaltimer() - t0 > kWaitBudgetNs) {
      set_status(status, RICI_ERR_TIMEOUT);
      *(volatile int *)abort_flag = 1;
      return false;
    }
    __nanosleep(32);
  }
}

// Bounded wait used while tearing down: no abort flag, a short budget (copies and MMAs that are
// still in flight after an abort finish within microseconds unless the GPU itself is stuck).
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, int *status) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > kDrainBudgetNs) {
      set_status(status, RICI_ERR_TIMEOUT);
      return;
    }
    __nanosleep(32);
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused with 128B swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4)                      // D format F32
                            | (0u << 7) | (0u << 10)       // A, B format F16
                            | ((uint32_t)(kBN >> 3) << 17) // N / 8
                            | ((uint32_t)(kBM >> 4) << 24);// M / 16

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- operand encoding (S2)

// One warp per image (launch-wide index).  Needle rows: [m | a]; haystack rows: [b^2 | -2b]
// (fp16, K = 2 N^2).  Also: the class flag (wide = outside the fp16 class, see the exactness
// note above), the list of wide images, and for needles A_i.
__global__ void k_tc_encode(const SearchScene *__restrict__ tab, const int *__restrict__ scene_of,
                            int64_t n, int N, int needle_side, __half *__restrict__ op,
                            int *__restrict__ wide_flag, int *__restrict__ wide_list,
                            int *__restrict__ wide_count, int *__restrict__ asum,
                            uint32_t *__restrict__ valid_mask, const int *__restrict__ skip_tile,
                            const int *__restrict__ any_tile) {
  const int lane = threadIdx.x & 31;
  // operand rows no tile will load are not written (the classes are still computed): needle
  // rows of skipped needle tiles, and every haystack row when no needle tile is left
  const bool hay_written = needle_side || !any_tile || *any_tile != 0;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int K0 = N * N;
  for (int64_t i = w; i < n; i += nw) {
    const SearchScene &sc = tab[scene_of[i]];
    const uint16_t *img = needle_side ? sc.needles + (i - sc.qoff) * K0
                                      : sc.haystack + (i - sc.hoff) * K0;
    __half *row = op + i * (int64_t)(2 * K0);
    const int lim = needle_side ? kNarrowA : kNarrowB;
    int wide = 0, a2 = 0, s1 = 0;  // needles: a2 = sum a^2; haystack: a2 = S2_j, s1 = S1_j
    const bool write = needle_side ? !(skip_tile && skip_tile[i / kBM]) : hay_written;
    for (int k0 = lane * 8; k0 < K0; k0 += 32 * 8) {
      __align__(16) __half lo[8], hi[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        const int r = k / N, c = k - r * N;
        const int d = c == 0 ? 0 : (int)img[r * N + c] - (int)img[r * N + c - 1];
        const bool nar = d >= -lim && d <= lim;
        wide |= !nar;
        const int dc = nar ? d : 0;
        a2 += dc * dc;
        if (needle_side) {
          lo[e] = __int2half_rn(dc != 0 ? 1 : 0);
          hi[e] = __int2half_rn(dc);
        } else {
          s1 += dc < 0 ? -dc : dc;
          lo[e] = __int2half_rn(dc * dc);
          hi[e] = __int2half_rn(-2 * dc);
        }
      }
      if (write) {
        *reinterpret_cast<int4 *>(row + k0) = *reinterpret_cast<int4 *>(lo);
        *reinterpret_cast<int4 *>(row + K0 + k0) = *reinterpret_cast<int4 *>(hi);
      }
    }
    wide = __any_sync(0xffffffffu, wide);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      a2 += __shfl_down_sync(0xffffffffu, a2, d);
      s1 += __shfl_down_sync(0xffffffffu, s1, d);
    }
    if (lane == 0) {
      if (!needle_side && (int64_t)a2 + 2ll * kNarrowA * s1 >= kExactSum) wide = 1;
      wide_flag[i] = wide;
      if (wide) wide_list[atomicAdd(wide_count, 1)] = (int)i;
      if (asum) asum[i] = a2;
      if (valid_mask && !wide) atomicOr(&valid_mask[i >> 5], 1u << (i & 31));
    }
  }
}

// ---------------------------------------------------------------- GEMM + rank epilogue (S3, S5)

struct TcArgs {
  const SearchScene *tab;
  int num_scenes;
  int64_t tiles;                  // all scenes' tiles
  int KT;                         // 2 N^2
  const int *nwide;               // needle wide flags (TC class)
  const int *nflags;              // per-needle state (0 = searchable)
  const int *asum;                // A_i
  const int64_t *dtrue;           // d(i, match_i)
  const uint32_t *hvalid;         // bit j: haystack image j is narrow
  int *rank;
  unsigned long long *best;
  int *status;
  int withhold_first_load;  // test hook: CTA 0 never issues its first stage (its waits time out)
  int group_m;              // needle tiles per group of the tile order
  const int *skip_needle;   // optional: 1 = this needle is ranked by another form
  const int *skip_tile;     // optional (single scene): 1 = needle tile m has no needle here
  const int *any_tile;      // with skip_tile: 0 = every tile is skipped (the grid returns at once)
};

// Tiles and their order: search_tile_of (common.cuh).
__device__ __forceinline__ TcTile tile_of(const SearchScene *tab, int ns, int64_t t, int group_m) {
  return search_tile_of(tab, ns, t, group_m);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_rank(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
              TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled stages
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *sA = smem;
  unsigned char *sB = smem + kStages * kStageA;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kStages * kStageB);
  uint64_t *empty = full + kStages;
  uint64_t *tfull = empty + kStages;
  uint64_t *tempty = tfull + 2;
  uint64_t *drain = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  // nothing to rank: return before any barrier, TMEM or TMA work (uniform over the grid)
  if (a.any_tile && *a.any_tile == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles = a.tiles;
  const int kblocks = a.KT / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const TcTile tt = tile_of(a.tab, a.num_scenes, t, a.group_m);
        if (a.skip_tile && a.skip_tile[tt.m]) continue;  // every role skips the same tiles
        const int ya = (int)(tt.qbeg + tt.m * kBM), yb = (int)(tt.hbeg + tt.n * kBN);
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const uint32_t s = it % kStages, round = it / kStages;
          if (!mbar_wait(&empty[s], (round & 1) ^ 1, a.status, abort_flag)) {
            ok = false;
            break;
          }
          if (a.withhold_first_load && blockIdx.x == 0 && it == 0) continue;
          mbar_arrive_expect_tx(&full[s], kStageA + kStageB);
          tma_load_2d(sA + s * kStageA, &map_a, &full[s], kb * kBK, ya);
          tma_load_2d(sB + s * kStageB, &map_b, &full[s], kb * kBK, yb);
        }
      }
      // Loads issued in the last kStages iterations may be unconsumed after an abort: wait for
      // them before the CTA exits (already-complete phases return at once).
      for (uint32_t j = 1; j <= (uint32_t)kStages && j <= it; ++j) {
        const uint32_t i = it - j;
        if (a.withhold_first_load && blockIdx.x == 0 && i == 0) continue;
        mbar_drain(&full[i % kStages], (i / kStages) & 1, a.status);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        if (a.skip_tile && a.skip_tile[tile_of(a.tab, a.num_scenes, t, a.group_m).m]) continue;
        const uint32_t buf = lt & 1, use = lt >> 1;
        ++lt;  // local count of processed tiles (selects the accumulator buffer)
        if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, a.status, abort_flag)) break;
        tc_fence_after();
        const uint32_t tacc = tmem + buf * kBN;
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const uint32_t s = it % kStages, round = it / kStages;
          if (!mbar_wait(&full[s], round & 1, a.status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + s * kStageA), b0 = smem_u32(sB + s * kStageB);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            tc_mma(tacc, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32),
                   (kb > 0 || kk > 0) ? 1u : 0u);
          }
          tc_commit(&empty[s]);  // frees the stage once these MMAs have read it
        }
        if (!ok) break;
        tc_commit(&tfull[buf]);  // accumulator ready for the epilogue
      }
      // every MMA this thread issued has finished before TMEM is released
      tc_commit(drain);
      mbar_drain(drain, 0, a.status);
    }
  } else {
    // ---------------- epilogue: warps 2..5, TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    uint32_t lt = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
      const TcTile tt = tile_of(a.tab, a.num_scenes, t, a.group_m);
      if (a.skip_tile && a.skip_tile[tt.m]) continue;
      const uint32_t buf = lt & 1, use = lt >> 1;
      ++lt;
      // warp-uniform outcome before the .sync.aligned TMEM loads
      const bool ready = __all_sync(0xffffffffu, mbar_wait(&tfull[buf], use & 1, a.status, abort_flag));
      if (!ready) break;
      tc_fence_after();
      const int64_t il = tt.m * kBM + row;  // scene-local needle
      const int64_t i = tt.qbeg + il;         // launch-wide needle
      const bool row_ok = il < tt.Q && a.nflags[i] == 0 && !a.nwide[i] &&
                          !(a.skip_needle && a.skip_needle[i]);
      float thr = 0.0f;
      int64_t asum = 0, thr_i = 0;
      if (row_ok) {
        asum = a.asum[i];
        thr_i = a.dtrue[i] - asum;
        // fp16-class S values are integers with |S| < 2^24; clamping keeps S < thr exact
        thr = (float)(thr_i > (1ll << 25) ? (1ll << 25) : (thr_i < -(1ll << 25) ? -(1ll << 25) : thr_i));
      }
      int cnt = 0;
      unsigned long long bestk = kNoBestTc;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + buf * kBN;
#pragma unroll 1
      for (int c0 = 0; c0 < kBN; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(taddr + c0, v);
        const int64_t j0 = tt.n * kBN + c0;  // scene-local haystack column
        uint32_t vm = 0;  // bit e: column j0 + e is a narrow haystack image of this scene
        if (row_ok && j0 < tt.H) {
          const int64_t g0 = tt.hbeg + j0;   // launch-wide index (any alignment)
          const uint32_t lo = a.hvalid[g0 >> 5], hi = a.hvalid[(g0 >> 5) + 1];
          const int sh = (int)(g0 & 31);
          vm = sh ? (lo >> sh) | (hi << (32 - sh)) : lo;
          const int64_t rem = tt.H - j0;
          if (rem < 32) vm &= (1u << rem) - 1u;
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const float sv = __uint_as_float(v[e]);
          const bool ok = (vm >> e) & 1u;
          cnt += (ok && sv < thr);
          if (ok && sv <= thr) {
            const unsigned long long dist = (unsigned long long)(asum + (int64_t)sv);
            const unsigned long long key = (dist << 32) | (unsigned long long)(uint32_t)(j0 + e);
            bestk = key < bestk ? key : bestk;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      if (row_ok) {
        if (cnt) atomicAdd(&a.rank[i], cnt);
        if (bestk != kNoBestTc) atomicMin(&a.best[i], bestk);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_map(CUtensorMap *map, const void *base, int64_t rows, int KT, int box_rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  cuuint64_t dims[2] = {(cuuint64_t)KT, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)KT * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool tc_supported(int N) { return N == 8 || N == 16 || N == 32 || N == 64 || N == 128; }

int64_t tc_workspace_bytes(int64_t Q, int64_t H, int N) {
  const int64_t KT = 2ll * N * N;
  Carver c(nullptr);
  c.take<__half>(Q * KT);
  c.take<__half>(H * KT);
  c.take<int>(Q);                 // A_i
  c.take<uint32_t>((H + 31) / 32 + 2);
  return c.off + 256;
}

cudaError_t launch_tc_encode_and_rank(const SearchScene *tab, int num_scenes, const int *qscene,
                                      const int *hscene, int64_t Q, int64_t H,
                                      int64_t tiles_total, int N, void *ws, int *nwide, int *hwide,
                                      int *wn_list, int *wh_list, int *counts,
                                      const int *nflags, const int64_t *dtrue, int *rank,
                                      unsigned long long *best, int *status, int test_withhold,
                                      cudaStream_t st, const int *skip_needle,
                                      const int *skip_tile, const int *any_tile) {
  const int64_t KT = 2ll * N * N;
  Carver c(ws);
  __half *opa = c.take<__half>(Q * KT);
  __half *opb = c.take<__half>(H * KT);
  int *asum = c.take<int>(Q);
  uint32_t *hvalid = c.take<uint32_t>((H + 31) / 32 + 2);
  cudaError_t e;
  if ((e = cudaMemsetAsync(hvalid, 0, sizeof(uint32_t) * ((H + 31) / 32 + 2), st)) != cudaSuccess)
    return e;
  auto blocks_for = [](int64_t warps) {
    int64_t b = (warps + 7) / 8;
    return (int)(b < 152 * 64 ? (b > 0 ? b : 1) : 152 * 64);
  };
  k_tc_encode<<<blocks_for(Q), 256, 0, st>>>(tab, qscene, Q, N, 1, opa, nwide, wn_list, counts + 0,
                                             asum, nullptr, skip_tile, nullptr);
  k_tc_encode<<<blocks_for(H), 256, 0, st>>>(tab, hscene, H, N, 0, opb, hwide, wh_list, counts + 1,
                                             nullptr, hvalid, nullptr, skip_tile ? any_tile : nullptr);
  count_launches(2);
  if (tiles_total == 0) return cudaGetLastError();
  CUtensorMap ma, mb;
  if ((e = encode_map(&ma, opa, Q, (int)KT, kBM)) != cudaSuccess) return e;
  if ((e = encode_map(&mb, opb, H, (int)KT, kBN)) != cudaSuccess) return e;
  TcArgs a;
  a.tab = tab;
  a.num_scenes = num_scenes;
  a.tiles = tiles_total;
  a.KT = (int)KT;
  a.nwide = nwide;
  a.nflags = nflags;
  a.asum = asum;
  a.dtrue = dtrue;
  a.hvalid = hvalid;
  a.rank = rank;
  a.best = best;
  a.status = status;
  a.withhold_first_load = test_withhold;
  a.group_m = current_tuning().tc_group_m;
  a.skip_needle = skip_needle;
  a.skip_tile = skip_tile;
  a.any_tile = skip_tile ? any_tile : nullptr;
  const size_t smem = 1024 + kStages * (kStageA + kStageB) + 256;
  if ((e = cudaFuncSetAttribute(k_tc_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(tiles_total < sms ? tiles_total : sms);
  k_tc_rank<<<grid, kTcThreads, smem, st>>>(ma, mb, a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace rici
