// Exact clutter-resistant search on the integer tensor cores (warp-level mma.sync s8, sm_103a).
//
// The distance of Eq. distanceFunctionExpression splits as in the fp16 tensor-core form:
//   d(i,j) = sum_k m_ik (a_ik - b_jk)^2 = A_i + S_ij,
//   A_i = sum_k a_ik^2,   S_ij = sum_k m_ik b_jk^2 - 2 a_ik b_jk,
// with a, b the column deltas (delta of column 0 := 0) and m_ik = [a_ik != 0].  Here every
// operand is an int8 and every product is accumulated in int32 by mma.sync m16n8k32:
//   G1 = sum_k a_ik b_jk,   G2 = sum_k m_ik q_jk,   G3 = sum_k m_ik r_jk,
// where b^2 = 128 q + r splits the squared haystack delta into two 7-bit limbs
// (q = b^2 >> 7 <= 126, r = b^2 & 127), so that  S_ij = 128 G2 + G3 - 2 G1.
//
// Exactness: for images whose deltas all satisfy |delta| <= 127 ("int8-narrow") every operand
// is an int8 value, |G1| <= 4032 * 127^2 < 2^26, 0 <= G2 <= 4032 * 126, 0 <= G3 <= 4032 * 127,
// so every int32 accumulation and |S| < 2^28 are exact.  Pairs with a wider side go to the exact
// int64 CUDA-core kernel, as in the other forms.  The rank test S_ij < d(i,match_i) - A_i and the
// top-1 key (A_i + S_ij, j) are evaluated in the epilogue; S is never written to memory.
//
// Work order: the tiles of the fp16 tensor-core form (128 needles x 256 haystack images, grouped
// along the needles for L2 reuse, every scene of a batch), each split into four 64 x 128 blocks
// of 8 warps (2 along the needles x 4 along the haystack, 32 x 32 pairs per warp).  Operands
// stream through a 4-stage cp.async pipeline of 64-byte K slices with an XOR swizzle of the
// 16-byte chunks, read by ldmatrix without bank conflicts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rici {
namespace {

constexpr int kI8BM = 64;        // needles per block
constexpr int kI8BN = 128;       // haystack images per block
constexpr int kI8KC = 64;        // bytes of K per pipeline stage
constexpr int kI8Stages = 4;
constexpr int kI8Threads = 256;  // 8 warps
constexpr int kI8StageBytes = (2 * kI8BM + 3 * kI8BN) * kI8KC;  // a, m + b, q, r: 32 KB
constexpr int kI8Narrow = 127;   // |delta| limit of the int8 operands

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of 16-byte chunk `chunk` (0..3) of row `row` in a [rows][64] byte tile: chunks are
// XOR-swizzled by row pair, so the 8 rows an ldmatrix phase reads fall in distinct banks.
__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)(row * kI8KC + ((chunk ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// D += A (16x32, row) * B (32x8, col), s8 x s8 -> s32.
__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- operand encoding (S1, S2)

// One warp per image (launch-wide index).  Needles: rows a (deltas) and m ([a != 0]) and A_i;
// haystack: rows b (deltas), q = b^2 >> 7 and r = b^2 & 127.  Every row is K0 = N^2 int8 values
// (position r * N + c, delta of column 0 := 0).  Images with a delta outside [-127, 127] are
// flagged wide and listed; their rows are not used.
__global__ void k_i8_encode(const SearchScene *__restrict__ tab, const int *__restrict__ scene_of,
                            int64_t n, int N, int needle_side, int8_t *__restrict__ o0,
                            int8_t *__restrict__ o1, int8_t *__restrict__ o2,
                            int *__restrict__ wide_flag, int *__restrict__ wide_list,
                            int *__restrict__ wide_count, int *__restrict__ asum) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int K0 = N * N;
  for (int64_t i = w; i < n; i += nw) {
    const SearchScene &sc = tab[scene_of[i]];
    const uint16_t *img = needle_side ? sc.needles + (i - sc.qoff) * K0
                                      : sc.haystack + (i - sc.hoff) * K0;
    int wide = 0, a2 = 0;
    for (int k0 = lane * 16; k0 < K0; k0 += 32 * 16) {
      __align__(16) int8_t v0[16], v1[16], v2[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int k = k0 + e;
        const int r = k / N, c = k - r * N;
        const int d = c == 0 ? 0 : (int)img[r * N + c] - (int)img[r * N + c - 1];
        const bool nar = d >= -kI8Narrow && d <= kI8Narrow;
        wide |= !nar;
        const int dc = nar ? d : 0;
        if (needle_side) {
          v0[e] = (int8_t)dc;
          v1[e] = (int8_t)(dc != 0);
          a2 += dc * dc;
        } else {
          const int sq = dc * dc;
          v0[e] = (int8_t)dc;
          v1[e] = (int8_t)(sq >> 7);
          v2[e] = (int8_t)(sq & 127);
        }
      }
      const int64_t off = i * (int64_t)K0 + k0;
      *reinterpret_cast<int4 *>(o0 + off) = *reinterpret_cast<const int4 *>(v0);
      *reinterpret_cast<int4 *>(o1 + off) = *reinterpret_cast<const int4 *>(v1);
      if (!needle_side) *reinterpret_cast<int4 *>(o2 + off) = *reinterpret_cast<const int4 *>(v2);
    }
    wide = __any_sync(0xffffffffu, wide);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) a2 += __shfl_down_sync(0xffffffffu, a2, d);
    if (lane == 0) {
      wide_flag[i] = wide;
      if (wide) wide_list[atomicAdd(wide_count, 1)] = (int)i;
      if (asum) asum[i] = a2;
    }
  }
}

// ---------------------------------------------------------------- GEMM + rank epilogue (S3, S5)

struct I8Args {
  const SearchScene *tab;
  int num_scenes;
  int group_m;
  int K0;                       // N^2
  const int8_t *na, *nm;        // needle rows [Qtot][K0]
  const int8_t *hb, *hq, *hr;   // haystack rows [Htot][K0]
  const int *nwide, *hwide;     // int8 class flags (1: some |delta| > 127)
  const int *nflags;            // per-needle state (0 = searchable)
  const int *asum;              // A_i
  const int64_t *dtrue;         // d(i, match_i)
  int *rank;
  unsigned long long *best;
};

__global__ void __launch_bounds__(kI8Threads, 1) k_i8_rank(I8Args a) {
  extern __shared__ __align__(128) unsigned char i8_smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;  // warp tile: needles wm*32.., haystack wn*32..
  const int64_t cta = blockIdx.x;
  const TcTile tt = search_tile_of(a.tab, a.num_scenes, cta >> 2, a.group_m);
  const int sub = (int)(cta & 3);
  const int64_t m0 = tt.m * 128 + (sub >> 1) * kI8BM;  // scene-local first needle
  const int64_t n0 = tt.n * 256 + (sub & 1) * kI8BN;   // scene-local first haystack image
  if (m0 >= tt.Q || n0 >= tt.H) return;  // uniform over the block

  // rows this thread copies: needle row tid/4 (arrays a, m), haystack rows tid/4 and tid/4 + 64
  // (arrays b, q, r); chunk tid % 4 of each 64-byte slice
  const int crow = tid >> 2, cchunk = tid & 3;
  const int64_t gq = tt.qbeg + min(m0 + crow, tt.Q - 1);
  const int64_t gh0 = tt.hbeg + min(n0 + crow, tt.H - 1);
  const int64_t gh1 = tt.hbeg + min(n0 + crow + 64, tt.H - 1);
  const int K0 = a.K0;
  const int8_t *pa = a.na + gq * K0 + cchunk * 16, *pm = a.nm + gq * K0 + cchunk * 16;
  const int8_t *pb0 = a.hb + gh0 * K0 + cchunk * 16, *pb1 = a.hb + gh1 * K0 + cchunk * 16;
  const int8_t *pq0 = a.hq + gh0 * K0 + cchunk * 16, *pq1 = a.hq + gh1 * K0 + cchunk * 16;
  const int8_t *pr0 = a.hr + gh0 * K0 + cchunk * 16, *pr1 = a.hr + gh1 * K0 + cchunk * 16;
  const uint32_t sbase = smem_addr(i8_smem);
  // stage layout: a [64][64], m [64][64], b [128][64], q [128][64], r [128][64]
  constexpr uint32_t kOffM = kI8BM * kI8KC, kOffB = 2 * kI8BM * kI8KC;
  constexpr uint32_t kOffQ = kOffB + kI8BN * kI8KC, kOffR = kOffQ + kI8BN * kI8KC;
  const uint32_t sw_a = swz(crow, cchunk), sw_b1 = swz(crow + 64, cchunk);
  auto load_stage = [&](int slot, int kc) {
    const uint32_t s = sbase + slot * kI8StageBytes;
    const int64_t ko = (int64_t)kc * kI8KC;
    cp_async16(s + sw_a, pa + ko);
    cp_async16(s + kOffM + sw_a, pm + ko);
    cp_async16(s + kOffB + sw_a, pb0 + ko);
    cp_async16(s + kOffB + sw_b1, pb1 + ko);
    cp_async16(s + kOffQ + sw_a, pq0 + ko);
    cp_async16(s + kOffQ + sw_b1, pq1 + ko);
    cp_async16(s + kOffR + sw_a, pr0 + ko);
    cp_async16(s + kOffR + sw_b1, pr1 + ko);
  };

  int g1[2][4][4], g2[2][4][4], g3[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) g1[mt][nt][e] = g2[mt][nt][e] = g3[mt][nt][e] = 0;

  // ldmatrix lane roles: matrix mi = lane / 8, row rr = lane % 8 within it
  const int mi = lane >> 3, rr = lane & 7;
  const int nk = K0 / kI8KC;
#pragma unroll
  for (int s = 0; s < kI8Stages - 1; ++s) {
    if (s < nk) load_stage(s, s);
    cp_async_commit();
  }
#pragma unroll 1
  for (int kc = 0; kc < nk; ++kc) {
    cp_async_wait<kI8Stages - 2>();
    __syncthreads();
    const int nxt = kc + kI8Stages - 1;
    if (nxt < nk) load_stage(nxt % kI8Stages, nxt);
    cp_async_commit();
    const uint32_t s = sbase + (kc % kI8Stages) * kI8StageBytes;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {  // two k32 steps per 64-byte slice
      uint32_t fa[2][4], fm[2][4], fb[4][2], fq[4][2], fr[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // A 16x32: matrices (rows 0-7, k 0-15), (rows 8-15, k 0-15), (0-7, 16-31), (8-15, 16-31)
        const int row = wm * 32 + mt * 16 + (mi & 1) * 8 + rr;
        const uint32_t o = swz(row, 2 * ks + (mi >> 1));
        ldsm_x4(s + o, fa[mt]);
        ldsm_x4(s + kOffM + o, fm[mt]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        // two n8 tiles: matrices (tile 2np, k 0-15), (2np, 16-31), (2np+1, 0-15), (2np+1, 16-31)
        const int row = wn * 32 + np * 16 + (mi >> 1) * 8 + rr;
        const uint32_t o = swz(row, 2 * ks + (mi & 1));
        uint32_t t4[4];
        ldsm_x4(s + kOffB + o, t4);
        fb[2 * np][0] = t4[0]; fb[2 * np][1] = t4[1]; fb[2 * np + 1][0] = t4[2]; fb[2 * np + 1][1] = t4[3];
        ldsm_x4(s + kOffQ + o, t4);
        fq[2 * np][0] = t4[0]; fq[2 * np][1] = t4[1]; fq[2 * np + 1][0] = t4[2]; fq[2 * np + 1][1] = t4[3];
        ldsm_x4(s + kOffR + o, t4);
        fr[2 * np][0] = t4[0]; fr[2 * np][1] = t4[1]; fr[2 * np + 1][0] = t4[2]; fr[2 * np + 1][1] = t4[3];
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma_s8(g1[mt][nt], fa[mt], fb[nt][0], fb[nt][1]);
          mma_s8(g2[mt][nt], fm[mt], fq[nt][0], fq[nt][1]);
          mma_s8(g3[mt][nt], fm[mt], fr[nt][0], fr[nt][1]);
        }
    }
  }
  cp_async_wait<0>();

  // ---- epilogue: accumulator (row g or g + 8 of an m16 tile, columns 2 tig, 2 tig + 1 of an n8)
  const int g = lane >> 2, tig = lane & 3;
  uint32_t colok = 0;  // bit nt*2 + e: column usable (inside the scene, int8-narrow)
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int64_t jl = n0 + wn * 32 + nt * 8 + tig * 2 + e;
      if (jl < tt.H && !a.hwide[tt.hbeg + jl]) colok |= 1u << (nt * 2 + e);
    }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t il = m0 + wm * 32 + mt * 16 + h * 8 + g;
      const int64_t i = tt.qbeg + il;
      const bool row_ok = il < tt.Q && a.nflags[i] == 0 && !a.nwide[i];
      int64_t asum = 0, thr = 0;
      if (row_ok) {
        asum = a.asum[i];
        thr = a.dtrue[i] - asum;
      }
      int cnt = 0;
      unsigned long long bestk = ~0ull;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int q = h * 2 + e;
          const int64_t S = 128 * (int64_t)g2[mt][nt][q] + g3[mt][nt][q] - 2 * (int64_t)g1[mt][nt][q];
          const bool ok = row_ok && ((colok >> (nt * 2 + e)) & 1u);
          cnt += (ok && S < thr);
          if (ok && S <= thr) {
            const int64_t jl = n0 + wn * 32 + nt * 8 + tig * 2 + e;
            const unsigned long long key =
                ((unsigned long long)(asum + S) << 32) | (unsigned long long)(uint32_t)jl;
            bestk = key < bestk ? key : bestk;
          }
        }
      cnt += __shfl_xor_sync(0xffffffffu, cnt, 1);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, 2);
      unsigned long long o = __shfl_xor_sync(0xffffffffu, bestk, 1);
      bestk = o < bestk ? o : bestk;
      o = __shfl_xor_sync(0xffffffffu, bestk, 2);
      bestk = o < bestk ? o : bestk;
      if (tig == 0 && row_ok) {
        if (cnt) atomicAdd(&a.rank[i], cnt);
        if (bestk != ~0ull) atomicMin(&a.best[i], bestk);
      }
    }
}

}  // namespace

bool i8_supported(int N) { return N == 8 || N == 16 || N == 32 || N == 64 || N == 128; }

int64_t i8_workspace_bytes(int64_t Q, int64_t H, int N) {
  const int64_t K0 = (int64_t)N * N;
  Carver c;
  c.take<int8_t>(Q * K0);  // a
  c.take<int8_t>(Q * K0);  // m
  c.take<int8_t>(H * K0);  // b
  c.take<int8_t>(H * K0);  // q
  c.take<int8_t>(H * K0);  // r
  c.take<int>(Q);          // A_i
  return c.off + 256;
}

cudaError_t launch_i8_encode_and_rank(const SearchScene *tab, int num_scenes, const int *qscene,
                                      const int *hscene, int64_t Q, int64_t H,
                                      int64_t tiles_total, int N, void *ws, int *nwide, int *hwide,
                                      int *wn_list, int *wh_list, int *counts,
                                      const int *nflags, const int64_t *dtrue, int *rank,
                                      unsigned long long *best, cudaStream_t st) {
  const int64_t K0 = (int64_t)N * N;
  Carver c(ws);
  int8_t *na = c.take<int8_t>(Q * K0);
  int8_t *nm = c.take<int8_t>(Q * K0);
  int8_t *hb = c.take<int8_t>(H * K0);
  int8_t *hq = c.take<int8_t>(H * K0);
  int8_t *hr = c.take<int8_t>(H * K0);
  int *asum = c.take<int>(Q);
  auto blocks_for = [](int64_t warps) {
    int64_t b = (warps + 7) / 8;
    return (int)(b < 152 * 64 ? (b > 0 ? b : 1) : 152 * 64);
  };
  k_i8_encode<<<blocks_for(Q), 256, 0, st>>>(tab, qscene, Q, N, 1, na, nm, nullptr, nwide, wn_list,
                                             counts + 0, asum);
  k_i8_encode<<<blocks_for(H), 256, 0, st>>>(tab, hscene, H, N, 0, hb, hq, hr, hwide, wh_list,
                                             counts + 1, nullptr);
  count_launches(2);
  if (tiles_total == 0) return cudaGetLastError();
  if (4 * tiles_total > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  I8Args a;
  a.tab = tab;
  a.num_scenes = num_scenes;
  a.group_m = current_tuning().tc_group_m;
  a.K0 = (int)K0;
  a.na = na;
  a.nm = nm;
  a.hb = hb;
  a.hq = hq;
  a.hr = hr;
  a.nwide = nwide;
  a.hwide = hwide;
  a.nflags = nflags;
  a.asum = asum;
  a.dtrue = dtrue;
  a.rank = rank;
  a.best = best;
  const int smem = kI8Stages * kI8StageBytes;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_i8_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
      cudaSuccess)
    return e;
  k_i8_rank<<<(unsigned)(4 * tiles_total), kI8Threads, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace rici
