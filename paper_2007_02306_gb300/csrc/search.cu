// Clutter-resistant search on sm_103a (Section 3.2: Listing 1, Eq. distanceFunctionExpression;
// ranking of Section 4.1 with the tie rule of Section 4.2).
//
// d(i, j) = sum over r in [0,N), c in [1,N) with a != 0 of (a - b)^2, a and b the needle's and
// haystack's column deltas.  rank_i = #{j : d(i,j) < d(i,match_i)}, top1_i = smallest j with
// minimal d(i,j).  Everything is integer arithmetic, so results are exact.
//
// Stages:
//   k_encode        per image: int8 column deltas (delta of column 0 := 0); for needles also
//                   a byte mask of the non-zero deltas and per-row sums of squared deltas, for
//                   the haystack a warp-interleaved layout (32 images per group, 16-byte chunks
//                   chunk-major); images with any |delta| > 127 are "wide" and listed apart.
//   k_true_distance d(i, match_i) in int64 straight from the uint16 images.
//   k_dense         narrow x narrow pairs on CUDA cores.  Per row, sum m(a-b)^2 =
//                   sum a^2 + sum (mb)^2 - 2 sum ab with sum a^2 precomputed and the other two
//                   as dp4a over 4 packed deltas (plus one AND for mb); each row's sum is >= 0,
//                   so partial sums are monotone and a pair stops once it exceeds
//                   d(i, match_i) (the early exit of Section 4.4, which never changes a rank).
//                   A block keeps 4 needles in shared memory and sweeps a band of haystack
//                   tiles (1,024 images each, four per thread at N <= 64), rows heaviest
//                   first; each broadcast needle word serves all of a thread's images.
//   k_wide          pairs with a wide side: Listing 1 over the needle's non-zero deltas in
//                   int64, reading the uint16 images.
//   k_finalize / k_top1_exact   combine counts and top-1 candidates.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"

namespace rici {
namespace {

constexpr int kDenseThreads = 256;     // threads of a dense block
constexpr int64_t kBandMax = 8;        // haystack tiles per band of the dense work order
constexpr int kWideThreads = 256;
constexpr unsigned long long kNoBest = ~0ull;

__device__ __forceinline__ int delta_at(const uint16_t *img, int N, int r, int c) {
  return c == 0 ? 0 : (int)img[r * N + c] - (int)img[r * N + c - 1];
}

// Byte offset of the delta at flat position k of image i in the warp-interleaved layout read by
// k_dense: 32 consecutive images form a group, and within a group each row is stored as chunks
// of CW 32-bit words per image, chunk-major, so the 32 lanes of a warp (32 consecutive images)
// read the same chunk of the same row with one contiguous 32 x 4CW-byte access.
__device__ __forceinline__ int64_t interleaved_offset(int64_t i, int N, int k) {
  const int WPR = N / 4, CW = WPR < 4 ? WPR : 4;
  const int r = k / N, c = k - r * N;
  const int w = c >> 2, v = w / CW, ww = w - v * CW;
  const int64_t g = i >> 5, l = i & 31;
  return ((((g * N + r) * (WPR / CW) + v) * 32 + l) * CW + ww) * 4 + (c & 3);
}

// Byte offset of the delta at flat position k of image i in the word-major layout read by
// k_sparse: 32 consecutive images form a group, and within a group word w (4 deltas) of the 32
// images is stored contiguously (128 bytes), so the 32 lanes of a warp reading the same word of
// their images make one coalesced access whatever the word.
__device__ __forceinline__ int64_t word_major_offset(int64_t i, int N, int k) {
  const int64_t g = i >> 5, l = i & 31;
  return ((g * (N * N / 4) + (k >> 2)) * 32 + l) * 4 + (k & 3);
}

// One warp per image.  interleave: 0 image-major deltas; 1 the layout of interleaved_offset (the
// haystack of the dense kernel); 2 the layout of word_major_offset (the haystack of k_sparse).
// row_sq (optional): per row, the sum of the squared (clamped) deltas, [n][N].
// list (optional): encode images list[0 .. *list_count) of imgs as images 0, 1, ... (a compacted
// subset, count read on the device; n is then an upper bound).
__global__ void k_encode(const uint16_t *__restrict__ imgs, int64_t n, int N,
                         int8_t *__restrict__ delta, int8_t *__restrict__ mask,
                         int *__restrict__ wide_flag, int *__restrict__ wide_list,
                         int *__restrict__ wide_count, int interleave, int *__restrict__ row_sq,
                         const int *__restrict__ list = nullptr,
                         const int *__restrict__ list_count = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int K = N * N;
  if (list) n = *list_count < n ? *list_count : n;
  // rows of a multiple of 32 positions: every pass of the warp lies in one row, so the row sums
  // of squared (clamped) deltas come from one warp reduction per pass
  const bool rows_by_pass = N % 32 == 0;
  for (int64_t i = w; i < n; i += nw) {
    const uint16_t *img = imgs + (list ? (int64_t)list[i] : i) * K;
    int wide = 0, row_acc = 0;
    for (int k = lane; k < K; k += 32) {
      int r = k / N, c = k - r * N;
      int d = delta_at(img, N, r, c);
      wide |= (d > 127 || d < -127);
      int dc = d > 127 ? 127 : (d < -127 ? -127 : d);
      const int64_t off = interleave == 1   ? interleaved_offset(i, N, k)
                          : interleave == 2 ? word_major_offset(i, N, k)
                                            : i * K + k;
      delta[off] = (int8_t)dc;
      if (mask) mask[i * K + k] = (int8_t)(d != 0 ? -1 : 0);
      if (row_sq && rows_by_pass) {
        row_acc += (int)__reduce_add_sync(0xffffffffu, (unsigned)(dc * dc));
        if (c - lane + 32 == N) {  // the row's last pass (uniform over the warp)
          if (lane == 0) row_sq[i * N + r] = row_acc;
          row_acc = 0;
        }
      }
    }
    if (row_sq && !rows_by_pass) {
      for (int r = lane; r < N; r += 32) {
        int sq = 0;
        for (int c = 1; c < N; ++c) {
          int d = delta_at(img, N, r, c);
          d = d > 127 ? 127 : (d < -127 ? -127 : d);
          sq += d * d;
        }
        row_sq[i * N + r] = sq;
      }
    }
    wide = __any_sync(0xffffffffu, wide);
    if (lane == 0) {
      wide_flag[i] = wide;
      if (wide) wide_list[atomicAdd(wide_count, 1)] = (int)i;
    }
  }
}

// Exact int64 distance of one pair, one warp.
__device__ int64_t warp_crss(const uint16_t *n, const uint16_t *h, int N) {
  const int lane = threadIdx.x & 31;
  long long s = 0;
  for (int k = lane; k < N * N; k += 32) {
    int r = k / N, c = k - r * N;
    if (c == 0) continue;
    int a = delta_at(n, N, r, c);
    if (a != 0) {
      long long d = (long long)a - (long long)delta_at(h, N, r, c);
      s += d * d;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  return __shfl_sync(0xffffffffu, s, 0);
}

__global__ void k_true_distance(const SearchScene *__restrict__ tab, const int *__restrict__ qscene,
                                int64_t Qtot, int N, int64_t *__restrict__ dtrue,
                                int *__restrict__ rank, unsigned long long *__restrict__ best,
                                int *__restrict__ flags, int *status) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t K = (int64_t)N * N;
  for (int64_t i = w; i < Qtot; i += nw) {
    const SearchScene &sc = tab[qscene[i]];
    const int64_t il = i - sc.qoff;
    const int64_t m = sc.match ? sc.match[il] : il;
    if (m < 0 || m >= sc.H) {
      if (lane == 0) {
        set_status(status, RICI_ERR_INDEX_OUT_OF_RANGE);
        dtrue[i] = -1;
        rank[i] = -1;
        best[i] = kNoBest;
        flags[i] = 2;  // invalid: no search for this needle
      }
      continue;
    }
    int64_t d = warp_crss(sc.needles + il * K, sc.haystack + m * K, N);
    if (lane == 0) {
      dtrue[i] = d;
      rank[i] = 0;
      best[i] = kNoBest;
      flags[i] = 0;
    }
  }
}

// Scene of every launch-wide needle and haystack image.
__global__ void k_scene_index(const SearchScene *__restrict__ tab, int ns, int64_t Qtot,
                              int64_t Htot, int *__restrict__ qscene, int *__restrict__ hscene) {
  const int64_t n = Qtot > Htot ? Qtot : Htot;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    if (x < Qtot) {
      int lo = 0, hi = ns - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].qoff <= x) lo = mid; else hi = mid - 1;
      }
      qscene[x] = lo;
    }
    if (x < Htot) {
      int lo = 0, hi = ns - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].hoff <= x) lo = mid; else hi = mid - 1;
      }
      hscene[x] = lo;
    }
  }
}

constexpr int kFillChunk = 150;
struct SearchFill {
  SearchScene e[kFillChunk];
  int n;
};
__global__ void k_fill_search_table(SearchScene *dst, SearchFill f) {
  for (int i = threadIdx.x; i < f.n; i += blockDim.x) dst[i] = f.e[i];
}

__device__ __forceinline__ unsigned long long pack_best(int64_t d, int64_t j) {
  unsigned long long dd = d >= 0xffffffffll ? 0xffffffffull : (unsigned long long)d;
  return (dd << 32) | (unsigned long long)(uint32_t)j;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    unsigned long long o = __shfl_down_sync(0xffffffffu, v, d);
    v = o < v ? o : v;
  }
  return v;
}

// Narrow x narrow pairs.  Block: kTQ needles (deltas + masks in shared memory) x
// kDenseThreads * kImg haystack images (kImg per thread, in consecutive groups of 32).
template <int N, int kTQ, int kImg, bool kCount>
__global__ void __launch_bounds__(kDenseThreads, (N * kImg <= 64 ? 4 : 2) * 256 / kDenseThreads)
    k_dense(
    const int8_t *__restrict__ ndelta, const int8_t *__restrict__ nmask,
    const int *__restrict__ nrowsq, const int *__restrict__ nwide, int64_t Q,
    const int8_t *__restrict__ hdelta,
    const int *__restrict__ hwide, int64_t H, const int64_t *__restrict__ dtrue,
    const int *__restrict__ nflags, int *__restrict__ rank, unsigned long long *__restrict__ best,
    unsigned long long *__restrict__ counters, int64_t tile0, int64_t tiles_q, int64_t tiles_h,
    int64_t band_h, const int *__restrict__ hcount, const int *__restrict__ hmap,
    const int *__restrict__ gate) {
  // hcount (optional): the haystack holds *hcount images (H is then an upper bound); hmap
  // (optional): haystack image j is image hmap[j] of the caller's haystack (a compacted subset);
  // gate (optional): *gate == 0 means no needle is ranked here, and every block returns at once
  constexpr int WPR = N / 4;  // 32-bit words per row
  constexpr int K = N * N;
  extern __shared__ int2 am_raw[];  // [kTQ][K/4] (needle delta word, mask word)
  auto am = reinterpret_cast<int2(*)[K / 4]>(am_raw);
  __shared__ int thr_s[kTQ];
  __shared__ int act_s[kTQ];
  __shared__ int wrow[kTQ][N];     // sum of squared needle deltas per (needle, row)
  __shared__ int ord[N];           // rows by decreasing tile weight
  __shared__ unsigned rmask[N];    // needles of the tile with a non-zero delta in the row
  __shared__ int nrows_s;
  const int tid = threadIdx.x, lane = tid & 31;
  // Work order: bands of band_h haystack tiles.  A block holds one needle tile and sweeps the
  // haystack tiles of one band; consecutive blocks take consecutive needle tiles of the same band,
  // so a band's haystack images are read from DRAM once and reused from L2 by every needle tile,
  // and the needle tile's set-up (shared-memory fill, row order) is paid once per band.
  const int64_t L = tile0 + blockIdx.x;
  const int64_t band = L / tiles_q, qt = L - band * tiles_q;
  const int64_t h0 = band * band_h;
  const int64_t h1 = tiles_h - h0 < band_h ? tiles_h : h0 + band_h;
  const int64_t q0 = qt * kTQ;
  if (gate && *gate == 0) return;  // uniform over the grid
  if (hcount) {
    H = *hcount < H ? *hcount : H;
    if (h0 * (int64_t)(kDenseThreads * kImg) >= H) return;  // uniform over the block
  }

  bool act = false;
  if (tid < kTQ) {
    const int64_t q = q0 + tid;
    act = q < Q && nflags[q] == 0 && !nwide[q];
    int64_t t = act ? dtrue[q] : -1;
    thr_s[tid] = t > 0x7fffffffll ? 0x7fffffff : (int)t;
    act_s[tid] = act;
  }
  if (!__syncthreads_or(act)) return;  // no needle of this tile is ranked here
  for (int x = tid; x < kTQ * (K / 4); x += kDenseThreads) {
    int q = x / (K / 4), wd = x - q * (K / 4);
    int a = 0, m = 0;
    if (q0 + q < Q) {
      a = reinterpret_cast<const int *>(ndelta + (q0 + q) * K)[wd];
      m = reinterpret_cast<const int *>(nmask + (q0 + q) * K)[wd];
    }
    am[q][wd] = make_int2(a, m);
  }
  __syncthreads();
  // Rows are visited heaviest first so that distances pass the early-exit threshold sooner;
  // the sum is order independent, so the result is unchanged.  Rows where no needle of the
  // tile has a non-zero delta contribute nothing and are skipped.
  for (int x = tid; x < kTQ * N; x += kDenseThreads) {
    int q = x / N, r = x - q * N;
    wrow[q][r] = act_s[q] ? nrowsq[(q0 + q) * N + r] : 0;
  }
  __syncthreads();
  __shared__ int tile_w[N];
  if (tid < N) {
    int W = 0;
    unsigned msk = 0;
#pragma unroll
    for (int q = 0; q < kTQ; ++q) {
      W += wrow[q][tid];
      if (wrow[q][tid] > 0) msk |= 1u << q;
    }
    rmask[tid] = msk;
    tile_w[tid] = W;
  }
  __syncthreads();
  if (tid < N) {
    const int W = tile_w[tid];
    int rk = 0, nz = 0;
    for (int r2 = 0; r2 < N; ++r2) {
      const int W2 = tile_w[r2];
      rk += (W2 > W) || (W2 == W && r2 < tid);
      nz += W2 > 0;
    }
    ord[rk] = tid;
    if (tid == 0) nrows_s = nz;
  }
  __syncthreads();
  const int nrows = nrows_s;

  constexpr int kTile = kDenseThreads * kImg;  // haystack images per tile
  constexpr int CW = WPR < 4 ? WPR : 4;
  constexpr int64_t kGroupWords = (int64_t)N * WPR * 32;  // one group of 32 interleaved images
  const int warp = tid >> 5;
  for (int64_t ht = h0; ht < h1; ++ht) {
    // this thread's images: j0 + 32 k, k < kImg (a warp owns kImg consecutive groups of 32)
    const int64_t j0 = ht * kTile + (int64_t)warp * (32 * kImg) + lane;
    int acc[kImg][kTQ];  // partial distance minus the needle's true distance (exit once > 0)
    unsigned alive[kImg];
    unsigned inrange = 0;  // images of this thread inside the haystack (their rows are loaded)
#pragma unroll
    for (int k = 0; k < kImg; ++k) {
      const int64_t j = j0 + 32 * k;
      const bool valid = j < H && !hwide[j];
      if (j < H) inrange |= 1u << k;
      alive[k] = 0;
#pragma unroll
      for (int q = 0; q < kTQ; ++q) {
        acc[k][q] = -thr_s[q];
        if (valid && act_s[q]) alive[k] |= 1u << q;
      }
    }
    const int *hgrp = reinterpret_cast<const int *>(hdelta) + (j0 >> 5) * kGroupWords + lane * CW;
    unsigned long long pair_rows = 0, lane_slots = 0;
    int hw[kImg][WPR];
#pragma unroll
    for (int k = 0; k < kImg; ++k)
#pragma unroll
      for (int v = 0; v < WPR; ++v) hw[k][v] = 0;
    for (int i = 0; i < nrows; ++i) {
      unsigned any = 0;
#pragma unroll
      for (int k = 0; k < kImg; ++k) any |= alive[k];
      if (__ballot_sync(0xffffffffu, any != 0) == 0) break;
      const int r = ord[i];
      const unsigned rm = rmask[r];
      unsigned use[kImg], uor = 0;
#pragma unroll
      for (int k = 0; k < kImg; ++k) {
        use[k] = alive[k] & rm;
        uor |= use[k];
        if (kCount) pair_rows += __popc(use[k]);
      }
      const unsigned wuse = __reduce_or_sync(0xffffffffu, uor);  // needles any lane still needs
#pragma unroll
      for (int k = 0; k < kImg; ++k) {
        // every row of an image inside the haystack is loaded, even once its pairs have all
        // exited: a uniform load is cheaper than the divergent branch that would skip it
        if ((inrange >> k) & 1u) {
          const int *src = hgrp + k * kGroupWords + r * (WPR * 32);
#pragma unroll
          for (int v = 0; v < WPR / CW; ++v) {
            if constexpr (CW == 4) {
              const int4 x = *reinterpret_cast<const int4 *>(src + v * 32 * CW);
              hw[k][4 * v] = x.x;
              hw[k][4 * v + 1] = x.y;
              hw[k][4 * v + 2] = x.z;
              hw[k][4 * v + 3] = x.w;
            } else {
              const int2 x = *reinterpret_cast<const int2 *>(src + v * 32 * CW);
              hw[k][2 * v] = x.x;
              hw[k][2 * v + 1] = x.y;
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kTQ; ++q) {
        if (((wuse >> q) & 1u) == 0) continue;
        if (kCount) lane_slots += kImg;  // kImg warp-wide needle-row iterations (32 lane slots each)
        // row sum of m (a - b)^2 = sum a^2 + sum (m b)^2 - 2 sum a b, with sum a^2 precomputed;
        // the (m b)^2 chain starts from the running value, and one chain per term and image
        // suffices because the warps of the block hide the dp4a latency
        const int w = wrow[q][r];
        int sb[kImg], sa[kImg];
#pragma unroll
        for (int k = 0; k < kImg; ++k) {
          sb[k] = acc[k][q] + w;
          sa[k] = 0;
        }
        const int4 *amq = reinterpret_cast<const int4 *>(&am[q][r * WPR]);
#pragma unroll
        for (int v = 0; v < WPR; v += 2) {
          const int4 x = amq[v >> 1];  // (a_v, m_v, a_v+1, m_v+1)
#pragma unroll
          for (int k = 0; k < kImg; ++k) {
            const int b0 = hw[k][v], b1 = hw[k][v + 1];
            const int bm0 = b0 & x.y, bm1 = b1 & x.w;
            sb[k] = __dp4a(bm0, bm0, sb[k]);
            sa[k] = __dp4a(x.x, b0, sa[k]);
            sb[k] = __dp4a(bm1, bm1, sb[k]);
            sa[k] = __dp4a(x.z, b1, sa[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < kImg; ++k) {
          // an image whose pair has exited keeps computing with stale deltas; its value is
          // never read again, since only pairs still alive are counted
          acc[k][q] = sb[k] - 2 * sa[k];
          if (acc[k][q] > 0) alive[k] &= ~(1u << q);
        }
      }
    }
    // count and top-1 candidates (pairs that never exceeded the threshold hold exact values)
#pragma unroll
    for (int q = 0; q < kTQ; ++q) {
      if (!act_s[q]) continue;
      int c = 0;
      unsigned long long b = kNoBest;
#pragma unroll
      for (int k = 0; k < kImg; ++k) {
        const bool fin = (alive[k] >> q) & 1u;
        c += fin && acc[k][q] < 0;
        const int64_t jj = j0 + 32 * k;
        const unsigned long long bk =
            fin ? pack_best(acc[k][q] + thr_s[q], hmap ? (int64_t)hmap[jj] : jj) : kNoBest;
        b = bk < b ? bk : b;
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
      b = warp_min_u64(b);
      if (lane == 0) {
        if (c) atomicAdd(&rank[q0 + q], c);
        if (b != kNoBest) atomicMin(&best[q0 + q], b);
      }
    }
    if (kCount) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) pair_rows += __shfl_down_sync(0xffffffffu, pair_rows, d);
      if (lane == 0 && pair_rows) atomicAdd(counters, pair_rows);
      if (lane == 0 && lane_slots) atomicAdd(counters + 3, 32ull * lane_slots);
    }
  }
}

// Sparse-needle form.  Listing 1 only touches positions where the needle's delta is non-zero, so
// each needle is reduced to the list of its 32-bit words (4 deltas) holding a non-zero delta:
// entry = (a word, mask word, byte offset of the word in the word-major haystack group,
// sum of the word's squared deltas).  Each word adds m(a-b)^2 >= 0 over its 4 positions, so the
// partial sum may be compared with d(i, match_i) after any word; words are listed heaviest
// first (descending sum a^2, in 64 logarithmic classes) so that pairs pass the threshold sooner.
// The order decides only when a pair stops, never its result.
constexpr int kSparseWarps = 8;   // needles per block, one per warp
constexpr int kSparseImg = 4;     // haystack images per lane
constexpr int kSparseStep = 2;    // needle words per step over the first kSparseHead words
constexpr int kSparseHead = 4;
constexpr int kSparseStepLong = 4;  // needle words per step after them (loads of a step are in
                                    // flight together)
constexpr int64_t kSparseBandMax = 64;  // haystack tiles per band of the sparse work order

__device__ __forceinline__ int sparse_class(int wsq) {  // 0 = heaviest
  const int lg = 31 - __clz(wsq);
  const int frac = lg >= 2 ? (wsq >> (lg - 2)) & 3 : (wsq << (2 - lg)) & 3;
  return 63 - (4 * lg + frac);
}

// One warp per needle: the needle's non-zero words as sparse entries, heaviest class first
// (order inside a class is arbitrary).  ent: [Q][K/4] int4 slabs; ecount[i] = entries of i.
__global__ void __launch_bounds__(256) k_sparse_needles(const int8_t *__restrict__ nd,
                                                        const int8_t *__restrict__ nm, int64_t Q,
                                                        int N, int4 *__restrict__ ent,
                                                        int *__restrict__ ecount) {
  __shared__ int cls_n[8][64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int KW = N * N / 4;
  int *cnt = cls_n[wib];
  for (int64_t i = w0; i < Q; i += nw) {
    const int *a32 = reinterpret_cast<const int *>(nd + i * (int64_t)N * N);
    const int *m32 = reinterpret_cast<const int *>(nm + i * (int64_t)N * N);
    cnt[lane] = 0;
    cnt[lane + 32] = 0;
    __syncwarp();
    for (int w = lane; w < KW; w += 32) {
      const int a = a32[w];
      if (a != 0) atomicAdd(&cnt[sparse_class(__dp4a(a, a, 0))], 1);
    }
    __syncwarp();
    // exclusive scan of the 64 class sizes (two per lane)
    const int c0 = cnt[2 * lane], c1 = cnt[2 * lane + 1];
    int incl = c0 + c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    cnt[2 * lane] = incl - c0 - c1;
    cnt[2 * lane + 1] = incl - c1;
    __syncwarp();
    int4 *e = ent + i * (int64_t)KW;
    for (int w = lane; w < KW; w += 32) {
      const int a = a32[w];
      if (a != 0) {
        const int wsq = __dp4a(a, a, 0);
        const int pos = atomicAdd(&cnt[sparse_class(wsq)], 1);
        e[pos] = make_int4(a, m32[w], w * 128, wsq);
      }
    }
    if (lane == 0) ecount[i] = total;
    __syncwarp();
  }
}

// Narrow needles x narrow haystack images over the needles' sparse entries.  Block: kSparseWarps
// needles (one per warp) sweeping a band of haystack tiles of 32 * kSparseImg images; lane l of a
// warp holds images j0 + l + 32 k.  Per step the warp reads kSparseStep entries (the same address
// in every lane) and each lane gathers the entries' words of its images that are still alive
// (one coalesced 128-byte access per warp and image slot).
template <bool kCount>
__global__ void __launch_bounds__(kSparseWarps * 32) k_sparse(
    const int4 *__restrict__ ent, const int *__restrict__ ecount,
    const int *__restrict__ nwide, int64_t Q, const int8_t *__restrict__ hword,
    const int *__restrict__ hwide, int64_t H, int N, const int64_t *__restrict__ dtrue,
    const int *__restrict__ nflags, int *__restrict__ rank, unsigned long long *__restrict__ best,
    unsigned long long *__restrict__ counters, int64_t tile0, int64_t tiles_q, int64_t tiles_h,
    int64_t band_h) {
  constexpr int kTile = 32 * kSparseImg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t L = tile0 + blockIdx.x;
  const int64_t band = L / tiles_q, qt = L - band * tiles_q;
  const int64_t h0 = band * band_h;
  const int64_t h1 = tiles_h - h0 < band_h ? tiles_h : h0 + band_h;
  const int64_t q = qt * kSparseWarps + warp;
  if (q >= Q || nflags[q] != 0 || nwide[q]) return;  // the whole warp leaves; no block barrier follows
  const int64_t tq = dtrue[q];
  const int thr = tq > 0x7fffffffll ? 0x7fffffff : (int)tq;
  const int KW = N * N / 4;
  const int ne = ecount[q];
  const int4 *e = ent + q * (int64_t)KW;
  const int64_t gbytes = (int64_t)KW * 128;  // one group of 32 images
  unsigned long long pair_words = 0, lane_slots = 0;
  for (int64_t ht = h0; ht < h1; ++ht) {
    const int64_t j0 = ht * kTile + lane;
    int acc[kSparseImg];  // partial distance minus the needle's true distance (exit once > 0)
    unsigned alive = 0;
#pragma unroll
    for (int k = 0; k < kSparseImg; ++k) {
      const int64_t j = j0 + 32 * k;
      acc[k] = -thr;
      if (j < H && !hwide[j]) alive |= 1u << k;
    }
    const int8_t *hb = hword + (j0 >> 5) * gbytes + lane * 4;
    // steps of S entries from e0 while any image of the warp is alive; returns where it stopped
    auto steps = [&](auto step_tag, int e0, int e_end) {
      constexpr int S = decltype(step_tag)::value;
      for (; e0 < e_end; e0 += S) {
        if (__ballot_sync(0xffffffffu, alive != 0) == 0) return ne;
        int4 E[S];
#pragma unroll
        for (int u = 0; u < S; ++u)
          E[u] = e0 + u < ne ? e[e0 + u] : make_int4(0, 0, 0, 0);  // a zero entry adds nothing
        int b[S][kSparseImg];
#pragma unroll
        for (int u = 0; u < S; ++u)
#pragma unroll
          for (int k = 0; k < kSparseImg; ++k)
            b[u][k] = (alive >> k) & 1u
                          ? *reinterpret_cast<const int *>(hb + k * gbytes + E[u].z)
                          : 0;
        if (kCount) {
          const int n = ne - e0 < S ? ne - e0 : S;
          pair_words += (unsigned long long)__popc(alive) * n;
          lane_slots += (unsigned long long)kSparseImg * n;
        }
#pragma unroll
        for (int u = 0; u < S; ++u)
#pragma unroll
          for (int k = 0; k < kSparseImg; ++k) {
            // m (a - b)^2 over the word = sum a^2 + sum (m b)^2 - 2 sum a b
            const int bm = b[u][k] & E[u].y;
            const int sq = __dp4a(bm, bm, acc[k] + E[u].w);
            acc[k] = sq - 2 * __dp4a(E[u].x, b[u][k], 0);
          }
#pragma unroll
        for (int k = 0; k < kSparseImg; ++k)
          if (acc[k] > 0) alive &= ~(1u << k);  // images that have exited keep stale sums
      }
      return e0;
    };
    // short steps first (most pairs of sparse needles stop within a word or two), then longer
    // steps with more loads in flight for the pairs that go on
    const int e_mid = ne < kSparseHead ? ne : kSparseHead;
    const int e1 = steps(std::integral_constant<int, kSparseStep>(), 0, e_mid);
    steps(std::integral_constant<int, kSparseStepLong>(), e1, ne);
    int c = 0;
    unsigned long long bb = kNoBest;
#pragma unroll
    for (int k = 0; k < kSparseImg; ++k) {
      const bool fin = (alive >> k) & 1u;
      c += fin && acc[k] < 0;
      const unsigned long long bk = fin ? pack_best(acc[k] + thr, j0 + 32 * k) : kNoBest;
      bb = bk < bb ? bk : bb;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
    bb = warp_min_u64(bb);
    if (lane == 0) {
      if (c) atomicAdd(&rank[q], c);
      if (bb != kNoBest) atomicMin(&best[q], bb);
    }
  }
  if (kCount) {  // lane_slots is the same in every lane of the warp
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) pair_words += __shfl_down_sync(0xffffffffu, pair_words, d);
    if (lane == 0 && pair_words) atomicAdd(counters, pair_words);
    if (lane == 0 && lane_slots) atomicAdd(counters + 3, 32ull * lane_slots);
  }
}

// Pairs with a wide side, exact int64 (launch-wide indices; haystack restricted to the needle's
// scene).  List mode:
//   pass 0: needles = wide needle list, haystack = the needle's whole scene.
//   pass 1: needles = all needles that are not wide, haystack = wide images of the same scene.
//   pass 2: needles = all needles, haystack = the whole scene (reference path).
__global__ void __launch_bounds__(kWideThreads) k_wide(
    const SearchScene *__restrict__ tab, const int *__restrict__ qscene,
    const int *__restrict__ hscene, int64_t Qtot, int64_t Hmax, int N, int pass,
    const int *__restrict__ nwide, const int *__restrict__ wide_n_list,
    const int *__restrict__ wide_n_count, const int *__restrict__ wide_h_list,
    const int *__restrict__ wide_h_count, const int64_t *__restrict__ dtrue,
    const int *__restrict__ nflags, int *__restrict__ rank, unsigned long long *__restrict__ best,
    int *__restrict__ top1_flag, unsigned long long *__restrict__ counters,
    const int *__restrict__ sub_list, const int *__restrict__ sub_count) {
  // sub_list (optional, pass 1): iterate entries sub_list[0 .. *sub_count) of the wide haystack
  // list only (the images of that list outside the int8 class)
  extern __shared__ int2 nz[];  // (flat position, needle delta) of non-zero needle deltas
  __shared__ int nnz_s;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t K = (int64_t)N * N;
  const int64_t nq = pass == 0 ? *wide_n_count : Qtot;
  const int64_t nh = pass == 1 ? (sub_list ? *sub_count : *wide_h_count) : Hmax;
  const int64_t chunks = (nh + kWideThreads - 1) / kWideThreads;
  const int64_t items = nq * chunks;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t qi = it / chunks, ch = it - qi * chunks;
    const int64_t i = pass == 0 ? wide_n_list[qi] : qi;
    if (nflags[i] != 0 || (pass == 1 && nwide[i])) continue;  // uniform over the block
    const int si = qscene[i];
    const SearchScene &sc = tab[si];
    if (pass != 1 && ch * kWideThreads >= sc.H) continue;     // uniform over the block
    const int64_t il = i - sc.qoff;
    const uint16_t *n = sc.needles + il * K;
    // compact the needle's non-zero deltas (row-major order)
    __syncthreads();
    if (tid == 0) nnz_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < K; base += kWideThreads) {
      int k = (int)(base + tid);
      int a = 0;
      if (k < K) {
        int r = k / N, c = k - r * N;
        a = delta_at(n, N, r, c);
      }
      unsigned bal = __ballot_sync(0xffffffffu, a != 0);
      int wbase = 0;
      if (lane == 0) wbase = atomicAdd(&nnz_s, __popc(bal));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (a != 0) nz[wbase + __popc(bal & ((1u << lane) - 1u))] = make_int2(k, a);
    }
    __syncthreads();
    const int nnz = nnz_s;
    const int64_t thr = dtrue[i];
    const int64_t hj = ch * kWideThreads + tid;
    int64_t jl = -1;  // scene-local haystack index
    if (pass == 1) {
      if (hj < nh) {
        const int64_t jg = wide_h_list[sub_list ? sub_list[hj] : hj];
        if (hscene[jg] == si) jl = jg - sc.hoff;
      }
    } else if (hj < sc.H) {
      jl = hj;
    }
    int cnt = 0;
    unsigned long long b = kNoBest;
    unsigned long long npairs = 0, nterms = 0;
    if (jl >= 0) {
      const uint16_t *h = sc.haystack + jl * K;
      long long acc = 0;
      int e = 0;
      for (; e < nnz && acc <= thr; ++e) {
        int2 p = nz[e];
        long long d = (long long)p.y - ((long long)h[p.x] - (long long)h[p.x - 1]);
        acc += d * d;
      }
      npairs = 1;
      nterms = e;
      if (acc <= thr) {
        cnt = acc < thr;
        b = pack_best(acc, jl);
        if (acc >= 0xffffffffll) atomicOr(&top1_flag[i], 1);
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    b = warp_min_u64(b);
    if (counters) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        npairs += __shfl_down_sync(0xffffffffu, npairs, d);
        nterms += __shfl_down_sync(0xffffffffu, nterms, d);
      }
    }
    if (lane == 0) {
      if (cnt) atomicAdd(&rank[i], cnt);
      if (b != kNoBest) atomicMin(&best[i], b);
      if (counters && npairs) {
        atomicAdd(counters + 1, npairs);
        atomicAdd(counters + 2, nterms);
      }
    }
  }
}

// Per-needle choice of form (RICI_SEARCH_AUTO): a needle whose non-zero delta words are at most
// 1/kAutoSparseShare of its words goes to the sparse-needle form, every other int8-class needle
// to the fp16 tensor cores.  Writes the tensor-core skip flags (sparse_of), the exclusions of the
// dense middle pass (the sparse needles and those outside int8) and of the sparse kernel (the
// tensor-core needles and those outside int8).
constexpr int kAutoSparseShare = 4;

__global__ void k_auto_assign(const int *__restrict__ ecount, const int *__restrict__ n8wide,
                              int64_t Q, int KW, int *__restrict__ sparse_of,
                              int *__restrict__ excl_dense, int *__restrict__ excl_sparse) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int wide = n8wide[i];
    const int sp = !wide && (int64_t)ecount[i] * kAutoSparseShare <= KW;
    sparse_of[i] = sp;
    excl_dense[i] = wide || sp;
    excl_sparse[i] = wide || !sp;
  }
}

// skip_tile[m] = 1 when no needle of tensor-core needle tile m (128 needles) is ranked there;
// *any_tile (zeroed before) becomes 1 when some tile is left.
__global__ void k_auto_tiles(const int *__restrict__ excl_dense, int64_t Q, int64_t tiles_m,
                             int *__restrict__ skip_tile, int *__restrict__ any_tile) {
  const int lane = threadIdx.x & 31;
  for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; m < tiles_m;
       m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int any = 0;
    for (int k = lane; k < 128; k += 32) {
      const int64_t i = m * 128 + k;
      any |= i < Q && !excl_dense[i];
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) {
      skip_tile[m] = !any;
      if (any) atomicOr(any_tile, 1);
    }
  }
}

// Scene-local outputs: rank, true distance and top-1 (smallest index among minimal distances).
__global__ void k_finalize(const SearchScene *__restrict__ tab, const int *__restrict__ qscene,
                           int64_t Qtot, const int *__restrict__ rank,
                           const int64_t *__restrict__ dtrue, const unsigned long long *__restrict__ best,
                           const int *__restrict__ nflags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Qtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const SearchScene &sc = tab[qscene[i]];
    const int64_t il = i - sc.qoff;
    sc.rank[il] = rank[i];
    if (sc.dtrue) sc.dtrue[il] = dtrue[i];
    if (sc.top1)
      sc.top1[il] = (nflags[i] != 0 || best[i] == kNoBest)
                        ? -1 : (int32_t)(uint32_t)(best[i] & 0xffffffffull);
  }
}

// Needles whose best distance reached 2^32-1: exact (distance, index) minimum over the scene.
__global__ void __launch_bounds__(256) k_top1_exact(const SearchScene *__restrict__ tab,
                                                   const int *__restrict__ qscene, int64_t Qtot,
                                                   int N, const int *__restrict__ top1_flag,
                                                   const int *__restrict__ nflags) {
  __shared__ long long bd[8];
  __shared__ long long bj[8];
  const int64_t K = (int64_t)N * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t i = blockIdx.x; i < Qtot; i += gridDim.x) {
    if (!top1_flag[i] || nflags[i]) continue;
    const SearchScene &sc = tab[qscene[i]];
    const int64_t il = i - sc.qoff;
    long long md = 0x7fffffffffffffffll, mj = -1;
    for (int64_t j = warp; j < sc.H; j += 8) {
      long long d = warp_crss(sc.needles + il * K, sc.haystack + j * K, N);
      if (d < md) {
        md = d;
        mj = j;
      }
    }
    if (lane == 0) {
      bd[warp] = md;
      bj[warp] = mj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long d0 = bd[0], j0 = bj[0];
      for (int w = 1; w < 8; ++w)
        if (bd[w] < d0 || (bd[w] == d0 && bj[w] < j0)) {
          d0 = bd[w];
          j0 = bj[w];
        }
      if (sc.top1) sc.top1[il] = (int32_t)j0;
    }
    __syncthreads();
  }
}

// Full distance matrix (exact int64), one warp per pair.
__global__ void k_distances(const uint16_t *__restrict__ nimg, int64_t Q,
                            const uint16_t *__restrict__ himg, int64_t H, int N,
                            int64_t *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t K = (int64_t)N * N;
  for (int64_t p = w; p < Q * H; p += nw) {
    const int64_t i = p / H, j = p - i * H;
    int64_t d = warp_crss(nimg + i * K, himg + j * K, N);
    if (lane == 0) out[p] = d;
  }
}

bool dense_supported(int N) { return N == 8 || N == 16 || N == 32 || N == 64 || N == 128; }

template <int N>
cudaError_t launch_dense(const int8_t *nd, const int8_t *nm, const int *nrs, const int *nw, int64_t Q,
                         const int8_t *hd, const int *hw, int64_t H, const int64_t *dt,
                         const int *nf, int *rank, unsigned long long *best,
                         unsigned long long *counters, cudaStream_t st,
                         const int *hcount = nullptr, const int *hmap = nullptr,
                         const int *gate = nullptr) {
  // 4 needles x 4 haystack images per thread (N <= 64; 120 registers, two blocks of 256 threads
  // per SM) is the fastest measured shape: each broadcast needle word serves four images, and
  // the per-row bookkeeping is shared by 16 (needle, image) pairs
  constexpr int kTQ = N <= 64 ? 4 : 2;  // N = 128: 64 KB of needle tile, two blocks per SM
  constexpr int kImg = N <= 64 ? 4 : 1;
  const size_t smem = sizeof(int2) * kTQ * (N * N / 4);
  auto kern = counters ? k_dense<N, kTQ, kImg, true> : k_dense<N, kTQ, kImg, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t th = (H + kDenseThreads * kImg - 1) / (kDenseThreads * kImg);
  const int64_t tq = (Q + kTQ - 1) / kTQ;
  // bands as long as possible while the grid still gives every SM a few waves of blocks
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t band_h = th * tq / ((int64_t)sms * 2 * 4);
  band_h = band_h < 1 ? 1 : (band_h > kBandMax ? kBandMax : band_h);
  const int64_t total = (th + band_h - 1) / band_h * tq;
  constexpr int64_t kMaxGrid = 0x7fffffffll;
  for (int64_t t0 = 0; t0 < total; t0 += kMaxGrid) {
    const int64_t n = total - t0 < kMaxGrid ? total - t0 : kMaxGrid;
    kern<<<(unsigned)n, kDenseThreads, smem, st>>>(nd, nm, nrs, nw, Q, hd, hw, H, dt, nf, rank,
                                                   best, counters, t0, tq, th, band_h, hcount,
                                                   hmap, gate);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_sparse(const int4 *ent, const int *ecount, const int *nw, int64_t Q,
                          const int8_t *hd, const int *hw, int64_t H, int N, const int64_t *dt,
                          const int *nf, int *rank, unsigned long long *best,
                          unsigned long long *counters, cudaStream_t st) {
  auto kern = counters ? k_sparse<true> : k_sparse<false>;
  const int64_t th = (H + 32 * kSparseImg - 1) / (32 * kSparseImg);
  const int64_t tq = (Q + kSparseWarps - 1) / kSparseWarps;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // bands as long as possible while the grid still gives every SM several waves of blocks
  int64_t band_h = th * tq / ((int64_t)sms * 8 * 4);
  band_h = band_h < 1 ? 1 : (band_h > kSparseBandMax ? kSparseBandMax : band_h);
  const int64_t total = (th + band_h - 1) / band_h * tq;
  constexpr int64_t kMaxGrid = 0x7fffffffll;
  for (int64_t t0 = 0; t0 < total; t0 += kMaxGrid) {
    const int64_t n = total - t0 < kMaxGrid ? total - t0 : kMaxGrid;
    kern<<<(unsigned)n, kSparseWarps * 32, 0, st>>>(ent, ecount, nw, Q, hd, hw, H, N, dt, nf, rank,
                                                    best, counters, t0, tq, th, band_h);
    count_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace

void search_tiles(int64_t Q, int64_t H, int32_t *tiles_m, int32_t *tiles_n) {
  *tiles_m = (int32_t)((Q + 127) / 128);
  *tiles_n = (int32_t)((H + 255) / 256);
}

int64_t search_batch_workspace_bytes(int num_scenes, int64_t Q, int64_t H, int N, int mode) {
  const int64_t K = (int64_t)N * N;
  mode &= 0xff;
  const bool autom = mode == RICI_SEARCH_AUTO && num_scenes == 1 && tc_supported(N) &&
                     dense_supported(N);
  const bool tensor = (mode == RICI_SEARCH_TENSOR || mode == RICI_SEARCH_DEFAULT ||
                       mode == RICI_SEARCH_AUTO) && tc_supported(N);
  const bool i8 = mode == RICI_SEARCH_INT8_TC && i8_supported(N);
  const bool packed = !tensor && !i8 && mode != RICI_SEARCH_EXACT_SLOW && dense_supported(N);
  const bool sparse = packed && mode == RICI_SEARCH_SPARSE;
  const bool mid = tensor && num_scenes == 1 && dense_supported(N);
  Carver c(nullptr);
  c.take<SearchScene>(num_scenes);
  c.take<int>(Q);                        // scene of each needle
  c.take<int>(H);                        // scene of each haystack image
  c.take<int8_t>(packed || mid ? Q * K : 0);  // needle deltas (CUDA-core forms)
  c.take<int8_t>(packed || mid ? Q * K : 0);  // needle masks
  c.take<int>((packed && !sparse) || mid ? Q * N : 0);  // needle row sums of squared deltas
  c.take<int8_t>(packed || mid ? (H + 31) / 32 * 32 * K : 0);  // haystack deltas (groups of 32)
  c.take<int>(Q);                        // needle wide flags
  c.take<int>(H);                        // haystack wide flags
  c.take<int>(Q);                        // wide needle list
  c.take<int>(H);                        // wide haystack list
  c.take<int>(8);                        // list lengths
  c.take<int>(Q);                        // per-needle state flags
  c.take<int>(Q);                        // top-1 exact fallback flags
  c.take<unsigned long long>(Q);         // packed best (distance, index)
  c.take<int64_t>(Q);                    // true distances
  c.take<int>(Q);                        // ranks
  c.take<int4>(sparse || autom ? Q * (K / 4) : 0);  // sparse needle entries (a slab per needle)
  c.take<int>(sparse || autom ? Q : 0);  // sparse entries per needle
  c.take<char>(tensor ? tc_workspace_bytes(Q, H, N) : 0);
  c.take<char>(i8 ? i8_workspace_bytes(Q, H, N) : 0);
  c.take<int>(mid ? Q : 0);      // int8 class flags of the needles (dense middle pass)
  c.take<int>(mid ? H : 0);      // int8 class flags of the compacted haystack images
  c.take<int>(mid ? Q + H : 0);  // lists written by its encodes
  c.take<int8_t>(autom ? (H + 31) / 32 * 32 * K : 0);  // word-major haystack of the sparse form
  c.take<int>(autom ? H : 0);     // its int8 class flags
  c.take<int>(autom ? 3 * Q : 0);  // per-needle choice and the two exclusions
  c.take<int>(autom ? Q / 128 + 2 : 0);  // tensor-core needle tiles to skip
  return c.off + 256;
}

int64_t search_workspace_bytes(int64_t Q, int64_t H, int32_t N, int32_t mode) {
  return search_batch_workspace_bytes(1, Q, H, N, mode);
}

cudaError_t launch_search_batch(const SearchScene *scenes, const SearchBatch &b, void *ws,
                                cudaStream_t st, int64_t *out_distances) {
  const int64_t Q = b.Qtot, H = b.Htot;
  const int N = b.N;
  const int64_t K = (int64_t)N * N;
  if (Q == 0) return cudaSuccess;
  const int withhold = (b.mode & RICI_SEARCH_TEST_WITHHOLD_LOAD) ? 1 : 0;
  const int mode = b.mode & 0xff;
  // RICI_SEARCH_AUTO (single scene): each needle ranked by the fp16 tensor cores or by the
  // sparse-needle form, chosen from its share of non-zero delta words (k_auto_assign)
  const bool autom = mode == RICI_SEARCH_AUTO && b.num_scenes == 1 && tc_supported(N) &&
                     dense_supported(N);
  const bool tensor = (mode == RICI_SEARCH_TENSOR || mode == RICI_SEARCH_DEFAULT ||
                       mode == RICI_SEARCH_AUTO) && tc_supported(N);
  const bool i8 = mode == RICI_SEARCH_INT8_TC && i8_supported(N);
  const bool packed = !tensor && !i8 && mode != RICI_SEARCH_EXACT_SLOW && dense_supported(N) &&
                      b.num_scenes == 1;
  const bool sparse = packed && mode == RICI_SEARCH_SPARSE;
  const bool dense = packed && !sparse;
  // single-scene tensor-core calls: pairs of a narrow needle with a haystack image outside the
  // fp16 class but inside int8 (32 < |delta| <= 127) run on the dense CUDA-core kernel over a
  // compacted haystack instead of the int64 kernel
  const bool mid = tensor && b.num_scenes == 1 && dense_supported(N);
  Carver c(ws);
  SearchScene *tab = c.take<SearchScene>(b.num_scenes);
  int *qscene = c.take<int>(Q);
  int *hscene = c.take<int>(H);
  int8_t *nd = c.take<int8_t>(packed || mid ? Q * K : 0);
  int8_t *nm = c.take<int8_t>(packed || mid ? Q * K : 0);
  int *nrs = c.take<int>(dense || mid ? Q * N : 0);
  int8_t *hd = c.take<int8_t>(packed || mid ? (H + 31) / 32 * 32 * K : 0);
  int *nwide = c.take<int>(Q);
  int *hwide = c.take<int>(H);
  int *wn_list = c.take<int>(Q);
  int *wh_list = c.take<int>(H);
  int *counts = c.take<int>(8);
  int *nflags = c.take<int>(Q);
  int *t1flag = c.take<int>(Q);
  unsigned long long *best = c.take<unsigned long long>(Q);
  int64_t *dt = c.take<int64_t>(Q);
  int *rank = c.take<int>(Q);
  int4 *sent = c.take<int4>(sparse || autom ? Q * (K / 4) : 0);
  int *scount = c.take<int>(sparse || autom ? Q : 0);
  char *tc_ws = tensor ? c.take<char>(tc_workspace_bytes(Q, H, N)) : nullptr;
  char *i8_ws = i8 ? c.take<char>(i8_workspace_bytes(Q, H, N)) : nullptr;
  int *mid_nflag = c.take<int>(mid ? Q : 0);
  int *mid_hflag = c.take<int>(mid ? H : 0);
  int *mid_list = c.take<int>(mid ? Q + H : 0);
  int8_t *hword = c.take<int8_t>(autom ? (H + 31) / 32 * 32 * K : 0);
  int *auto_hflag = c.take<int>(autom ? H : 0);
  int *auto_n = c.take<int>(autom ? 3 * Q : 0);
  int *skip_tile = c.take<int>(autom ? Q / 128 + 2 : 0);
  int *sparse_of = autom ? auto_n : nullptr;
  int *excl_dense = autom ? auto_n + Q : nullptr;
  int *excl_sparse = autom ? auto_n + 2 * Q : nullptr;

  cudaError_t e;
  for (int s0 = 0; s0 < b.num_scenes; s0 += kFillChunk) {
    SearchFill f;
    f.n = b.num_scenes - s0 < kFillChunk ? b.num_scenes - s0 : kFillChunk;
    for (int i = 0; i < f.n; ++i) f.e[i] = scenes[s0 + i];
    k_fill_search_table<<<1, 256, 0, st>>>(tab + s0, f);
    count_launches(1);
  }
  if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * 8, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t1flag, 0, sizeof(int) * Q, st)) != cudaSuccess) return e;
  const int wpb = 8;
  auto blocks_for = [&](int64_t items) {
    int64_t nb = (items + wpb - 1) / wpb;
    return (int)(nb < 152 * 64 ? (nb > 0 ? nb : 1) : 152 * 64);
  };
  k_scene_index<<<blocks_for((Q > H ? Q : H) / 32 + 1), 256, 0, st>>>(tab, b.num_scenes, Q, H,
                                                                      qscene, hscene);
  k_true_distance<<<blocks_for(Q), 32 * wpb, 0, st>>>(tab, qscene, Q, N, dt, rank, best, nflags,
                                                       b.status);
  count_launches(2);
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(b.counters);
  const size_t wide_smem = sizeof(int2) * (size_t)K;
  if ((e = cudaFuncSetAttribute(k_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)wide_smem)) != cudaSuccess)
    return e;
  auto wide = [&](int pass, const int *sub_list = nullptr, const int *sub_count = nullptr) {
    k_wide<<<152 * 8, kWideThreads, wide_smem, st>>>(tab, qscene, hscene, Q, b.Hmax, N, pass,
                                                   nwide, wn_list, counts + 0, wh_list,
                                                   counts + 1, dt, nflags, rank, best, t1flag, cnt,
                                                   sub_list, sub_count);
    count_launches(1);
  };
  auto run_dense = [&](const int *nexcl, const int *hexcl, const int *hcount, const int *hmap,
                       const int *gate = nullptr) {
    switch (N) {
      case 8: return launch_dense<8>(nd, nm, nrs, nexcl, Q, hd, hexcl, H, dt, nflags, rank, best, cnt, st, hcount, hmap, gate);
      case 16: return launch_dense<16>(nd, nm, nrs, nexcl, Q, hd, hexcl, H, dt, nflags, rank, best, cnt, st, hcount, hmap, gate);
      case 32: return launch_dense<32>(nd, nm, nrs, nexcl, Q, hd, hexcl, H, dt, nflags, rank, best, cnt, st, hcount, hmap, gate);
      case 64: return launch_dense<64>(nd, nm, nrs, nexcl, Q, hd, hexcl, H, dt, nflags, rank, best, cnt, st, hcount, hmap, gate);
      default: return launch_dense<128>(nd, nm, nrs, nexcl, Q, hd, hexcl, H, dt, nflags, rank, best, cnt, st, hcount, hmap, gate);
    }
  };
  if (tensor) {
    const SearchScene &s0 = scenes[0];
    if (mid) {
      // CUDA-core encode of every needle (the fp16-class ones are int8-class too)
      k_encode<<<blocks_for(Q), 32 * wpb, 0, st>>>(s0.needles, Q, N, nd, nm, mid_nflag, mid_list,
                                                   counts + 2, 0, nrs);
      count_launches(1);
    }
    if (autom) {
      // each needle's form, decided before the tensor-core kernel runs
      k_sparse_needles<<<blocks_for(Q), 32 * wpb, 0, st>>>(nd, nm, Q, N, sent, scount);
      k_auto_assign<<<blocks_for(Q / 32 + 1), 256, 0, st>>>(scount, mid_nflag, Q, (int)(K / 4),
                                                            sparse_of, excl_dense, excl_sparse);
      k_auto_tiles<<<blocks_for(Q / 128 + 1), 256, 0, st>>>(excl_dense, Q, (Q + 127) / 128,
                                                            skip_tile, counts + 5);
      count_launches(3);
    }
    if ((e = launch_tc_encode_and_rank(tab, b.num_scenes, qscene, hscene, Q, H, b.tiles_total, N,
                                       tc_ws, nwide, hwide, wn_list, wh_list, counts, nflags, dt,
                                       rank, best, b.status, withhold, st, sparse_of,
                                       autom ? skip_tile : nullptr, counts + 5)) != cudaSuccess)
      return e;
    wide(0);  // needles outside the fp16 class against the whole haystack (int64)
    if (mid) {
      // the haystack images outside the fp16 class, compacted in list order (list and count
      // from the tensor-core encode); narrow needles x those images on CUDA cores, and the
      // int64 kernel only for the compacted images outside the int8 class
      k_encode<<<blocks_for(H), 32 * wpb, 0, st>>>(s0.haystack, H, N, hd, nullptr, mid_hflag,
                                                   mid_list + Q, counts + 3, 1, nullptr, wh_list,
                                                   counts + 1);
      count_launches(1);
      // (AUTO: counts[5] = 0 when no needle is left for the tensor-core side)
      if ((e = run_dense(autom ? excl_dense : nwide, mid_hflag, counts + 1, wh_list,
                         autom ? counts + 5 : nullptr)) != cudaSuccess)
        return e;
      // the compacted encode listed its images outside the int8 class (compact indices)
      wide(1, mid_list + Q, counts + 3);
    } else {
      wide(1);
    }
    if (autom) {
      // the sparse-needle form for its needles against every int8-class image (the encode's list
      // of images outside int8 goes to wh_list, whose readers above precede it on the stream)
      k_encode<<<blocks_for(H), 32 * wpb, 0, st>>>(s0.haystack, H, N, hword, nullptr, auto_hflag,
                                                   wh_list, counts + 4, 2, nullptr);
      count_launches(1);
      if ((e = launch_sparse(sent, scount, excl_sparse, Q, hword, auto_hflag, H, N, dt, nflags,
                             rank, best, cnt, st)) != cudaSuccess)
        return e;
    }
  } else if (i8) {
    if ((e = launch_i8_encode_and_rank(tab, b.num_scenes, qscene, hscene, Q, H, b.tiles_total, N,
                                       i8_ws, nwide, hwide, wn_list, wh_list, counts, nflags, dt,
                                       rank, best, st)) != cudaSuccess)
      return e;
    wide(0);
    wide(1);
  } else if (dense) {
    // single scene: launch-wide indices are the scene's own
    const SearchScene &s0 = scenes[0];
    k_encode<<<blocks_for(Q), 32 * wpb, 0, st>>>(s0.needles, Q, N, nd, nm, nwide, wn_list,
                                                 counts + 0, 0, nrs);
    k_encode<<<blocks_for(H), 32 * wpb, 0, st>>>(s0.haystack, H, N, hd, nullptr, hwide, wh_list,
                                                 counts + 1, 1, nullptr);
    count_launches(2);
    if ((e = run_dense(nwide, hwide, nullptr, nullptr)) != cudaSuccess) return e;
    wide(0);
    wide(1);
  } else if (sparse) {
    const SearchScene &s0 = scenes[0];
    k_encode<<<blocks_for(Q), 32 * wpb, 0, st>>>(s0.needles, Q, N, nd, nm, nwide, wn_list,
                                                 counts + 0, 0, nullptr);
    k_encode<<<blocks_for(H), 32 * wpb, 0, st>>>(s0.haystack, H, N, hd, nullptr, hwide, wh_list,
                                                 counts + 1, 2, nullptr);
    k_sparse_needles<<<blocks_for(Q), 32 * wpb, 0, st>>>(nd, nm, Q, N, sent, scount);
    count_launches(3);
    if ((e = launch_sparse(sent, scount, nwide, Q, hd, hwide, H, N, dt, nflags, rank, best, cnt,
                           st)) != cudaSuccess)
      return e;
    wide(0);
    wide(1);
  } else {
    if ((e = cudaMemsetAsync(nwide, 0, sizeof(int) * Q, st)) != cudaSuccess) return e;
    wide(2);
  }
  k_finalize<<<blocks_for(Q * wpb), 256, 0, st>>>(tab, qscene, Q, rank, dt, best, nflags);
  k_top1_exact<<<(int)(Q < 152 * 8 ? Q : 152 * 8), 256, 0, st>>>(tab, qscene, Q, N, t1flag,
                                                                 nflags);
  count_launches(2);
  if (out_distances && b.num_scenes == 1) {
    k_distances<<<blocks_for(Q * H), 32 * wpb, 0, st>>>(scenes[0].needles, Q, scenes[0].haystack,
                                                         H, N, out_distances);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_search(const SearchArgs &a, void *ws, cudaStream_t st) {
  SearchScene sc = {};
  sc.needles = a.needles;
  sc.haystack = a.haystack;
  sc.match = a.true_match;
  sc.rank = a.out_rank;
  sc.dtrue = a.out_true_distance;
  sc.top1 = a.out_top1;
  sc.Q = a.num_needles;
  sc.H = a.num_haystack;
  search_tiles(sc.Q, sc.H, &sc.tiles_m, &sc.tiles_n);
  SearchBatch b;
  b.num_scenes = 1;
  b.Qtot = sc.Q;
  b.Htot = sc.H;
  b.Hmax = sc.H;
  b.tiles_total = (int64_t)sc.tiles_m * sc.tiles_n;
  b.N = a.resolution;
  b.mode = a.mode;
  b.counters = a.counters;
  b.status = a.status;
  return launch_search_batch(&sc, b, ws, st, a.out_distances);
}

}  // namespace rici
