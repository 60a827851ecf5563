// RICI generation on sm_103a (Section 3.1 of the paper).
//
// Pipeline per rici_generate call (all on the caller's stream, no host synchronisation):
//   1. k_tri_bbox     box of the triangles' bounding-sphere centres, per scene.
//   2. k_tri_bin      bounding sphere of every triangle; bin it by the Morton code of its centre
//                     on a 2^L grid over that box (8^L bins, L <= 7).
//   3. scan           bin counts -> bin starts.
//   4. k_tri_scatter  64-byte triangle records (sphere, FP32 vertices, global indices) in bin
//                     order: the records follow a space-filling curve, so runs of consecutive
//                     records are compact in space.
//   5. k_chunk_spheres  a bounding sphere of every run of 32 records (chunk) and of 1024
//                     records (group).
//   6. k_generate     one CTA per oriented point.  Its warps test the groups of the point's
//                     scene against the support cylinder, then the chunks of passing groups,
//                     then the records of passing chunks (a sphere fails only if every record
//                     in it fails), project the surviving triangles (Eqs.
//                     relativeLocation..secondRotation) and split the (triangle, layer) work
//                     evenly over the 32 lanes.  Each layer's single/double crossing radii
//                     (Section 3.1.2) become column intervals added to a shared-memory
//                     difference image, which is prefix summed, saturated and stored as packed
//                     uint16 (32- or 64-bit stores).
// The clutter measure and spin images (bottom of this file) bin triangles into a hashed uniform
// grid instead and scan the grid cells around each oriented point.
//
// Exactness: the FP32 path carries a forward error bound for every predicate (vertex side
// of a layer, |E|^2 against alpha^2, the signs of E0.D and E1.D, alpha^2 |D|^2 against
// (E0 x D)^2).  A (triangle, layer) whose predicate lies inside its bound is recomputed in
// FP64 with the definition's operation order (explicit _rn intrinsics, no contraction), so
// every count equals the FP64 definition bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace rici {
namespace {

constexpr float kU = 5.9604644775390625e-08f;  // 2^-24: unit roundoff of FP32
constexpr float kSafety = 2.0f;                // multiplies every derived error bound
constexpr uint32_t kSkip = 0xFFFFFFFEu;
constexpr float kCellClamp = 1048576.0f;  // |cell coordinate| limit (2^20)
constexpr int kSlot = 21;  // words per staged triangle (odd stride: conflict-free lookups)
constexpr int kScanItems = kGenScanItems;
constexpr int kGenMaxCellsPerReach = 4;      // generation: up to (2 x 4 + 1)^3 cells per point
constexpr int kClutterMaxCellsPerReach = 3;  // clutter measure and spin images: up to 7^3
// shared words per warp: candidate queue, FP64 queue (triangle records, then their layers as
// bytes), staged triangles
constexpr int kPerWarp = 64 + 64 + 16 + 32 * kSlot;

__host__ __device__ constexpr uint32_t bucket_count(int64_t nt) { return generate_bucket_count(nt); }

__device__ __forceinline__ int cell_coord(float x, float inv_cell) {
  float f = floorf(x * inv_cell);
  f = fminf(fmaxf(f, -kCellClamp), kCellClamp);
  return (int)f;
}

__device__ __forceinline__ uint32_t cell_hash(int ix, int iy, int iz, uint32_t mask) {
  return (((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u)) &
         mask;
}

// Order-preserving map of finite floats to int32 (a min / max of the ints is a min / max of the
// floats); the map is its own inverse.
__device__ __forceinline__ int float_order(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float order_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Bits of x (< 2^10) spread to every third position.
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

struct TriSphere {
  float cx, cy, cz, r;
};

// Bounding sphere of the triangle's AABB, inflated to cover rounding of centre and radius.
__device__ __forceinline__ TriSphere tri_sphere(const float v[9]) {
  float lx = fminf(fminf(v[0], v[3]), v[6]), hx = fmaxf(fmaxf(v[0], v[3]), v[6]);
  float ly = fminf(fminf(v[1], v[4]), v[7]), hy = fmaxf(fmaxf(v[1], v[4]), v[7]);
  float lz = fminf(fminf(v[2], v[5]), v[8]), hz = fmaxf(fmaxf(v[2], v[5]), v[8]);
  TriSphere s;
  s.cx = 0.5f * (lx + hx);
  s.cy = 0.5f * (ly + hy);
  s.cz = 0.5f * (lz + hz);
  float ex = 0.5f * (hx - lx), ey = 0.5f * (hy - ly), ez = 0.5f * (hz - lz);
  float cm = fmaxf(fabsf(s.cx), fmaxf(fabsf(s.cy), fabsf(s.cz)));
  s.r = sqrtf(ex * ex + ey * ey + ez * ez) * (1.0f + 1e-5f) + 1e-6f * cm + 1e-30f;
  return s;
}

struct GridParams {
  float inv_cell;
  float r_big;
  uint32_t mask;
};

// Scene of a launch-wide index: the last table entry whose offset is <= idx (entries with no
// items share their offset with the next one, so the match always owns idx).
__device__ __forceinline__ int scene_of_tri(const GenScene *tab, int ns, int64_t idx) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].tri_off <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int scene_of_origin(const GenScene *tab, int ns, int64_t idx) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].origin_off <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Box of the bounding-sphere centres of each scene's valid triangles (ints of float_order; the
// table fill sets every box empty).  Triangles with a bad index or a non-finite vertex are left
// to k_tri_bin, which reports them.  Warps whose triangles all belong to one scene reduce first.
__global__ void k_tri_bbox(const GenScene *__restrict__ tab, int ns, int64_t nt_total,
                           int *__restrict__ bbox) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); t0 < nt_total;
       t0 += stride) {
    const int64_t t = t0 + lane < nt_total ? t0 + lane : nt_total - 1;
    const int sidx = scene_of_tri(tab, ns, t);
    const GenScene &sc = tab[sidx];
    const int64_t tl = t - sc.tri_off;
    const int64_t nv = sc.nv;
    bool ok = t0 + lane < nt_total;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (ok) {
      int id[3] = {sc.tris[3 * tl], sc.tris[3 * tl + 1], sc.tris[3 * tl + 2]};
      ok = id[0] >= 0 && id[0] < nv && id[1] >= 0 && id[1] < nv && id[2] >= 0 && id[2] < nv;
      if (ok) {
        float v[9];
        for (int k = 0; k < 3; ++k)
          for (int d = 0; d < 3; ++d) {
            v[3 * k + d] = sc.V[3 * (int64_t)id[k] + d];
            ok = ok && isfinite(v[3 * k + d]);
          }
        if (ok) {
          const TriSphere ts_ = tri_sphere(v);
          lo[0] = hi[0] = ts_.cx;
          lo[1] = hi[1] = ts_.cy;
          lo[2] = hi[2] = ts_.cz;
        }
      }
    }
    const int s0 = __shfl_sync(0xffffffffu, sidx, 0);
    if (__all_sync(0xffffffffu, sidx == s0)) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], d));
          hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], d));
        }
      ok = lane == 0 && lo[0] <= hi[0];
    }
    if (ok) {
      int *bb = bbox + 8 * (int64_t)sidx;
      for (int k = 0; k < 3; ++k) {
        atomicMin(bb + k, float_order(lo[k]));
        atomicMax(bb + 3 + k, float_order(hi[k]));
      }
    }
  }
}

// Bins every triangle by its bounding sphere.  With bbox == nullptr (clutter measure, spin
// images): a hashed uniform grid of cell edge 1 / inv_cell, wide triangles in the scene's big
// list.  Otherwise (generation): every triangle by the Morton code of its centre on a 2^L grid
// over its scene's box of centres (8^L <= the scene's bucket count), so that records sorted by
// bucket follow a space-filling curve and runs of consecutive records are compact.
__global__ void k_tri_bin(const GenScene *__restrict__ tab, int ns, int64_t nt_total, GridParams g,
                          const int *__restrict__ bbox, int *__restrict__ counts,
                          uint32_t *__restrict__ tb, int *__restrict__ ts, int *status) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt_total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const GenScene &sc = tab[scene_of_tri(tab, ns, t)];
    const int64_t tl = t - sc.tri_off;
    const int64_t nv = sc.nv;
    int id[3] = {sc.tris[3 * tl], sc.tris[3 * tl + 1], sc.tris[3 * tl + 2]};
    if (id[0] < 0 || id[0] >= nv || id[1] < 0 || id[1] >= nv || id[2] < 0 || id[2] >= nv) {
      set_status(status, RICI_ERR_INDEX_OUT_OF_RANGE);
      tb[t] = kSkip;
      continue;
    }
    float v[9];
    bool fin = true;
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) {
        v[3 * k + d] = sc.V[3 * (int64_t)id[k] + d];
        fin = fin && isfinite(v[3 * k + d]);
      }
    if (!fin) {
      set_status(status, RICI_ERR_NONFINITE_INPUT);
      tb[t] = kSkip;
      continue;
    }
    TriSphere s = tri_sphere(v);
    uint32_t b = sc.nbuckets;  // the scene's big list
    if (bbox) {
      const int *bb = bbox + 8 * (int64_t)scene_of_tri(tab, ns, t);
      const float lo[3] = {order_float(bb[0]), order_float(bb[1]), order_float(bb[2])};
      const float ext = fmaxf(fmaxf(order_float(bb[3]) - lo[0], order_float(bb[4]) - lo[1]),
                              order_float(bb[5]) - lo[2]);
      const int L = (31 - __clz(sc.nbuckets)) / 3;
      const float top = (float)((1 << L) - 1);
      const float scale = (ext > 0.0f && ext < 1e30f) ? (float)(1 << L) / ext : 0.0f;
      const float c[3] = {s.cx, s.cy, s.cz};
      uint32_t q[3];
      for (int k = 0; k < 3; ++k) {
        const float f = scale > 0.0f ? floorf((c[k] - lo[k]) * scale) : 0.0f;
        q[k] = (uint32_t)fminf(fmaxf(f, 0.0f), top);
      }
      b = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    } else {
      const float lim = kCellClamp - 4.0f;
      bool big = s.r > g.r_big || !(fabsf(s.cx * g.inv_cell) < lim) ||
                 !(fabsf(s.cy * g.inv_cell) < lim) || !(fabsf(s.cz * g.inv_cell) < lim);
      if (!big)
        b = cell_hash(cell_coord(s.cx, g.inv_cell), cell_coord(s.cy, g.inv_cell),
                      cell_coord(s.cz, g.inv_cell), sc.nbuckets - 1);
    }
    const uint32_t gb = (uint32_t)(sc.bucket_off + b);
    tb[t] = gb;
    ts[t] = atomicAdd(&counts[gb], 1);
  }
}

__global__ void k_tri_scatter(const GenScene *__restrict__ tab, int ns, int64_t nt_total,
                              const uint32_t *__restrict__ tb, const int *__restrict__ ts,
                              const int *__restrict__ starts, float4 *__restrict__ rec) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt_total;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = tb[t];
    if (b == kSkip) continue;
    const GenScene &sc = tab[scene_of_tri(tab, ns, t)];
    const int64_t tl = t - sc.tri_off;
    const int64_t pos = (int64_t)starts[b] + ts[t];
    int id[3] = {sc.tris[3 * tl], sc.tris[3 * tl + 1], sc.tris[3 * tl + 2]};
    float v[9];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) v[3 * k + d] = sc.V[3 * (int64_t)id[k] + d];
    TriSphere s = tri_sphere(v);
    // four columns of nt_total records: the culling pass streams only the first (16 bytes per
    // triangle), the set-up of survivors reads the other three
    rec[pos] = make_float4(s.cx, s.cy, s.cz, s.r);
    rec[nt_total + pos] = make_float4(v[0], v[1], v[2], v[3]);
    rec[2 * nt_total + pos] = make_float4(v[4], v[5], v[6], v[7]);
    rec[3 * nt_total + pos] = make_float4(v[8], __int_as_float(id[0]), __int_as_float(id[1]),
                                          __int_as_float(id[2]));
  }
}

// Warp collective: a sphere containing every lane's sphere c (c.w < 0: none).  Returns w < 0 when
// no lane has one and an infinite radius when the result is not finite.  The centre is that of
// the box of the spheres; the radius is the largest |c - C| + c.w, raised to cover its rounding.
__device__ __forceinline__ float4 sphere_of_spheres(float4 c) {
  const bool v = c.w >= 0.0f;
  float lo[3] = {v ? c.x - c.w : INFINITY, v ? c.y - c.w : INFINITY, v ? c.z - c.w : INFINITY};
  float hi[3] = {v ? c.x + c.w : -INFINITY, v ? c.y + c.w : -INFINITY, v ? c.z + c.w : -INFINITY};
#pragma unroll
  for (int d = 16; d > 0; d >>= 1)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], d));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], d));
    }
  if (!__any_sync(0xffffffffu, v)) return make_float4(0.0f, 0.0f, 0.0f, -1.0f);
  const float Cx = 0.5f * (lo[0] + hi[0]), Cy = 0.5f * (lo[1] + hi[1]), Cz = 0.5f * (lo[2] + hi[2]);
  float e = 0.0f;
  if (v) {
    const float dx = c.x - Cx, dy = c.y - Cy, dz = c.z - Cz;
    e = sqrtf(dx * dx + dy * dy + dz * dz) + c.w;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, d));
  const float rho = e * (1.0f + 1e-5f) + 1e-6f * (fabsf(Cx) + fabsf(Cy) + fabsf(Cz)) + 1e-30f;
  if (!(isfinite(Cx) && isfinite(Cy) && isfinite(Cz) && rho < 1e30f))
    return make_float4(0.0f, 0.0f, 0.0f, INFINITY);
  return make_float4(Cx, Cy, Cz, rho);
}

constexpr int kChunkShift = 5;   // 32 records per chunk
constexpr int kGroupShift = 10;  // 32 chunks (1024 records) per group

// Bounding spheres of every 32-record chunk and every 1024-record group of the sorted records
// (*nrec of them), each containing the bounding spheres of its records; a chunk or group at a
// scene boundary covers the records of both scenes.  One block of 32 warps per group.
__global__ void __launch_bounds__(1024) k_chunk_spheres(const float4 *__restrict__ rec,
                                                        const int *__restrict__ nrec,
                                                        float4 *__restrict__ chk,
                                                        float4 *__restrict__ grp) {
  __shared__ float4 cs[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = *nrec;
  const int64_t g = blockIdx.x;
  const int64_t ci = (g << (kGroupShift - kChunkShift)) + w;
  const int64_t t = (ci << kChunkShift) + lane;
  float4 c = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
  if (t < n) c = rec[t];
  const float4 sc = sphere_of_spheres(c);
  if (lane == 0) {
    cs[w] = sc;
    if (sc.w >= 0.0f) chk[ci] = sc;
  }
  __syncthreads();
  if (w == 0) {
    const float4 gs = sphere_of_spheres(cs[lane]);
    if (lane == 0 && gs.w >= 0.0f) grp[g] = gs;
  }
}

// Writes up to kFillChunk scene-table entries passed by value (no host memory is read later) and
// sets their boxes of triangle centres empty.
constexpr int kFillChunk = 200;
struct GenFill {
  GenScene e[kFillChunk];
  int n;
};
__global__ void k_fill_gen_table(GenScene *dst, GenFill f, int *bbox) {
  for (int i = threadIdx.x; i < f.n; i += blockDim.x) {
    dst[i] = f.e[i];
    for (int k = 0; k < 3; ++k) {
      bbox[8 * i + k] = 0x7fffffff;
      bbox[8 * i + 3 + k] = (int)0x80000000;
    }
  }
}

// ------------------------------------------------------------------ exclusive scan (int32)

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? warp_sums[lane] : 0;
    int wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < nw) warp_sums[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  int r = warp_sums[warp] + x - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_partials(const int *__restrict__ in, int64_t n, int *__restrict__ partials) {
  __shared__ int ws[32];
  __shared__ int tot;
  int64_t base = (int64_t)blockIdx.x * kScanItems;
  int s = 0;
  for (int i = threadIdx.x; i < kScanItems; i += blockDim.x)
    if (base + i < n) s += in[base + i];
  block_exclusive_scan(s, ws, &tot);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void k_scan_top(int *partials, int nb) {
  __shared__ int ws[32];
  __shared__ int tot;
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? partials[i] : 0;
    int ex = block_exclusive_scan(v, ws, &tot);
    if (i < nb) partials[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[nb] = carry;
}

__global__ void k_scan_final(const int *__restrict__ in, int64_t n, const int *__restrict__ partials,
                             int *__restrict__ out) {
  __shared__ int ws[32];
  __shared__ int tot;
  const int per = kScanItems / 256;  // blockDim.x == 256
  int64_t base = (int64_t)blockIdx.x * kScanItems + threadIdx.x * per;
  int v[per];
  int s = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int run = partials[blockIdx.x] + block_exclusive_scan(s, ws, &tot);
#pragma unroll
  for (int k = 0; k < per; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = partials[gridDim.x];
}

// ------------------------------------------------------------------ generation kernel

struct KArgs {
  const GenScene *tab;
  int num_scenes;
  int64_t origin_base;  // first launch-wide origin index of this grid
  const float4 *rec;    // triangle records, 4 columns: rec[k * rs + t]
  int64_t rs;           // column stride of rec (the launch's triangle count)
  const int *starts;
  float inv_cell;
  float cell;       // grid cell edge (1 / inv_cell)
  float reach;      // support-sphere radius + largest small-triangle radius (+ margin)
  float R;
  int N;
  float alpha_cull;  // pretest radius limit (alpha_{N-1} plus margin)
  float beta_cull;   // pretest height limit (beta_{N-1} plus margin)
  int mode;
  int nhalf;        // neighbourhood half-width in cells (cell edge > reach / nhalf)
  float r_big;      // largest bounding radius of a binned triangle
  const float4 *chk;  // generation: bounding spheres of 32-record chunks of rec
  const float4 *grp;  // generation: bounding spheres of 1024-record groups of rec
  unsigned long long *counters;
  int *status;
};

struct Shared {
  int *diff;     // [N][N] difference image
  double *a2d;   // alpha_c^2 (FP64 definition)
  double *bd;    // beta_r (FP64 definition)
  float *a2f;    // alpha_c^2 rounded to FP32
  float *bf;     // beta_r rounded to FP32
  double *fr;    // S (3 doubles), Nax, Nay, Nbx, Nbz
  int *buckets;  // neighbour buckets ((2 nhalf + 1)^3 cells + the big list), then the first
                 // candidate of each
  int *bdup;     // 1: skip this entry (out of reach or repeated bucket), then the end of its
                 // candidate range (= its first candidate for a skipped entry)
  int *wq;       // this warp's candidate queue [64]
  int *wst;      // this warp's item-owner marks for the current 32 items [32] (aliases the first
                 // half of wq, which is free once a batch's triangles are staged)
  int *bq_rec;   // this warp's FP64 queue: triangle record [64]
  unsigned char *bq_r;  // this warp's FP64 queue: layer [64]
  float *slots;  // this warp's staged triangles [32][kSlot]
};

// slot layout (words)
enum {
  SX = 0, SY = 3, SZ = 6, SGID = 9, SDE = 12,
  SINV = 15,   // 1 / (z_j - z_i) of edge k (opposite vertex k, i < j local indices)
  SMETA = 18,  // first layer (bits 0-7), side-band layer of each vertex (bits 8-15, 16-23,
               // 24-31; kNoBand for none; kAllBand in bits 8-15: every layer goes to FP64)
  SREC = 19
};
constexpr unsigned kNoBand = 0xFF, kAllBand = 0xFE;

// Estimate of the number of columns c with alpha_c^2 <= x (alpha_c = R (2c+1) / 2N, so the count
// is floor(N sqrt(x) / R + 1/2)), in [0, N].  Off by one at most, and only within a few ulps of a
// column boundary: every caller then checks the margins to both neighbouring columns, a check that
// fails (sends the item to FP64) whenever the estimate is not the exact count.
__device__ __forceinline__ int count_estimate_f(float x, int N, float scale) {
  const float s = x > 0.0f ? x * rsqrtf(x) * scale : 0.0f;
  const float fc = floorf((s + 1.0f) * 0.5f);
  return (fc >= (float)N) ? N : ((fc > 0.0f) ? (int)fc : 0);
}

__device__ __forceinline__ int lower_count_d(double x, const double *a2d, int N) {
  // number of columns c with a2d[c] <= x (a2d strictly increasing)
  int lo = 0, hi = N;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a2d[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Eq. rotationCoefficients (second pair on the rotated x component) with the identity rule,
// in FP64 with the definition's operation order: fr = (Nax, Nay, Nbx, Nbz).
__device__ __forceinline__ void frame_fp64(float nxf, float nyf, float nzf, double *fr) {
  const double nx = nxf, ny = nyf, nz = nzf;
  const double h = __dsqrt_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)));
  double Nax = 1.0, Nay = 0.0;
  if (h != 0.0) {
    Nax = __ddiv_rn(nx, h);
    Nay = __ddiv_rn(ny, h);
  }
  const double n2x = __dadd_rn(__dmul_rn(Nax, nx), __dmul_rn(Nay, ny));
  const double g = __dsqrt_rn(__dadd_rn(__dmul_rn(n2x, n2x), __dmul_rn(nz, nz)));
  double Nbx = 0.0, Nbz = 1.0;
  if (g != 0.0) {
    Nbx = __ddiv_rn(n2x, g);
    Nbz = __ddiv_rn(nz, g);
  }
  fr[0] = Nax;
  fr[1] = Nay;
  fr[2] = Nbx;
  fr[3] = Nbz;
}

// Eqs. relativeLocation, firstRotation, secondRotation in FP32 with explicit roundings (the
// frame coefficients rounded to FP32).  Returns |dx| + |dy| + |dz|, the scale of the error bound
// |T32 - T64| <= 10 u (|dx| + |dy| + |dz|) used by the generation kernel.
__device__ __forceinline__ float project_fp32(float px, float py, float pz, float Sx, float Sy,
                                              float Sz, float fax, float fay, float fbx,
                                              float fbz, float &tx, float &ty, float &tz) {
  const float dx = __fsub_rn(px, Sx), dy = __fsub_rn(py, Sy), dz = __fsub_rn(pz, Sz);
  const float qx = __fmaf_rn(fay, dy, __fmul_rn(fax, dx));
  const float qy = __fmaf_rn(fax, dy, -__fmul_rn(fay, dx));
  tx = __fmaf_rn(fbz, qx, -__fmul_rn(fbx, dz));
  ty = qy;
  tz = __fmaf_rn(fbx, qx, __fmul_rn(fbz, dz));
  return fabsf(dx) + fabsf(dy) + fabsf(dz);
}

// Projection of n points into one oriented point's frame with the generation kernel's FP32
// stage (one thread per point; each computes the frame).
__global__ void k_project_fp32(const float *__restrict__ pts, int64_t n, const float *__restrict__ sv,
                               const float *__restrict__ sn, float *__restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double fr[4];
    frame_fp64(sn[0], sn[1], sn[2], fr);
    float tx, ty, tz;
    project_fp32(pts[3 * k], pts[3 * k + 1], pts[3 * k + 2], sv[0], sv[1], sv[2],
                 __double2float_rn(fr[0]), __double2float_rn(fr[1]), __double2float_rn(fr[2]),
                 __double2float_rn(fr[3]), tx, ty, tz);
    out[3 * k] = tx;
    out[3 * k + 1] = ty;
    out[3 * k + 2] = tz;
  }
}

__device__ __forceinline__ void project64(float px, float py, float pz, const double *fr,
                                          double T[3]) {
  double dx = __dsub_rn((double)px, fr[0]);
  double dy = __dsub_rn((double)py, fr[1]);
  double dz = __dsub_rn((double)pz, fr[2]);
  const double Nax = fr[3], Nay = fr[4], Nbx = fr[5], Nbz = fr[6];
  double qx = __dadd_rn(__dmul_rn(Nax, dx), __dmul_rn(Nay, dy));
  double qy = __dadd_rn(__dmul_rn(-Nay, dx), __dmul_rn(Nax, dy));
  T[0] = __dsub_rn(__dmul_rn(Nbz, qx), __dmul_rn(Nbx, dz));
  T[1] = qy;
  T[2] = __dadd_rn(__dmul_rn(Nbx, qx), __dmul_rn(Nbz, dz));
}

// FP64 evaluation of one (triangle, layer) with the definition's operation order.
// Returns false when the triangle does not cross the layer; otherwise the single-crossing
// columns are [lo, hi) and the double-crossing columns [dlo, lo).
// (Plain pointer arguments: no structure has to live in local memory.)
__device__ __forceinline__ bool layer_fp64(const float4 *__restrict__ recs, int64_t rs,
                                        const double *fr, const double *bd, const double *a2d,
                                        int N, int rec, int r, int &lo, int &hi, int &dlo) {
  float4 r1 = recs[rs + rec], r2 = recs[2 * rs + rec], r3 = recs[3 * rs + rec];
  double T[3][3];
  project64(r1.x, r1.y, r1.z, fr, T[0]);
  project64(r1.w, r2.x, r2.y, fr, T[1]);
  project64(r2.z, r2.w, r3.x, fr, T[2]);
  const int gid[3] = {__float_as_int(r3.y), __float_as_int(r3.z), __float_as_int(r3.w)};
  const double beta = bd[r];
  int s0 = T[0][2] >= beta, s1 = T[1][2] >= beta, s2 = T[2][2] >= beta;
  if (s0 == s1 && s1 == s2) return false;
  int lone = (s0 != s1 && s0 != s2) ? 0 : ((s1 != s0 && s1 != s2) ? 1 : 2);
  int oa = lone == 0 ? 1 : 0;
  int ob = lone == 2 ? 1 : 2;
  // crossed edges evaluated from the lower to the higher global vertex index
  int ua = gid[lone] < gid[oa] ? lone : oa, va = gid[lone] < gid[oa] ? oa : lone;
  int ub = gid[lone] < gid[ob] ? lone : ob, vb = gid[lone] < gid[ob] ? ob : lone;
  double la = __ddiv_rn(__dsub_rn(beta, T[ua][2]), __dsub_rn(T[va][2], T[ua][2]));
  double lb = __ddiv_rn(__dsub_rn(beta, T[ub][2]), __dsub_rn(T[vb][2], T[ub][2]));
  double Eax = __dadd_rn(T[ua][0], __dmul_rn(la, __dsub_rn(T[va][0], T[ua][0])));
  double Eay = __dadd_rn(T[ua][1], __dmul_rn(la, __dsub_rn(T[va][1], T[ua][1])));
  double Ebx = __dadd_rn(T[ub][0], __dmul_rn(lb, __dsub_rn(T[vb][0], T[ub][0])));
  double Eby = __dadd_rn(T[ub][1], __dmul_rn(lb, __dsub_rn(T[vb][1], T[ub][1])));
  bool swap = gid[ub] < gid[ua] || (gid[ub] == gid[ua] && gid[vb] < gid[va]);
  double E0x = swap ? Ebx : Eax, E0y = swap ? Eby : Eay;
  double E1x = swap ? Eax : Ebx, E1y = swap ? Eay : Eby;
  double e0 = __dadd_rn(__dmul_rn(E0x, E0x), __dmul_rn(E0y, E0y));
  double e1 = __dadd_rn(__dmul_rn(E1x, E1x), __dmul_rn(E1y, E1y));
  int c0 = lower_count_d(e0, a2d, N), c1 = lower_count_d(e1, a2d, N);
  lo = min(c0, c1);
  hi = max(c0, c1);
  dlo = lo;
  if (lo > 0) {
    double Dx = __dsub_rn(E1x, E0x), Dy = __dsub_rn(E1y, E0y);
    double d0 = __dadd_rn(__dmul_rn(E0x, Dx), __dmul_rn(E0y, Dy));
    double d1 = __dadd_rn(__dmul_rn(E1x, Dx), __dmul_rn(E1y, Dy));
    if (d0 < 0.0 && d1 > 0.0) {
      double cr = __dsub_rn(__dmul_rn(E0x, Dy), __dmul_rn(E0y, Dx));
      double dd = __dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy));
      double cr2 = __dmul_rn(cr, cr);
      // first column with alpha^2 * dd > cr^2 (monotone in the column)
      int l = 0, h = lo;
      while (l < h) {
        int mid = (l + h) >> 1;
        if (__dmul_rn(a2d[mid], dd) > cr2) h = mid; else l = mid + 1;
      }
      dlo = l;
    }
  }
  return true;
}

// FP32 evaluation with forward error bounds against the FP64 definition.
// Returns 0: no crossing, 1: intervals valid, 2: a predicate lies inside its error band
// (the caller re-evaluates the item in FP64).
__device__ __forceinline__ int layer_fp32(const float *__restrict__ bf, const float *__restrict__ a2f,
                                          int N, const float *sl, int r, float scale, int &lo,
                                          int &hi, int &dlo) {
  const float beta = bf[r];
  float tz0 = sl[SZ], tz1 = sl[SZ + 1], tz2 = sl[SZ + 2];
  int s0 = tz0 >= beta, s1 = tz1 >= beta, s2 = tz2 >= beta;
  if (s0 == s1 && s1 == s2) return 0;
  int lone = (s0 != s1 && s0 != s2) ? 0 : ((s1 != s0 && s1 != s2) ? 1 : 2);
  int oa = lone == 0 ? 1 : 0;
  int ob = lone == 2 ? 1 : 2;
  // slice the two crossed edges (lone, oa) and (lone, ob) in local vertex order: E lies within
  // the per-edge bound of the FP64 point whatever the orientation, so the FP32 path only has to
  // keep the roles of E0 and E1 (chosen by global vertex indices as in the definition)
  const int g_l = __float_as_int(sl[SGID + lone]), g_a = __float_as_int(sl[SGID + oa]),
            g_b = __float_as_int(sl[SGID + ob]);
  const int ia = min(lone, oa), ja = max(lone, oa);  // edge opposite ob
  const int ib = min(lone, ob), jb = max(lone, ob);  // edge opposite oa
  const float la = __fmul_rn(__fsub_rn(beta, sl[SZ + ia]), sl[SINV + ob]);
  const float lb = __fmul_rn(__fsub_rn(beta, sl[SZ + ib]), sl[SINV + oa]);
  float Eax = __fmaf_rn(la, __fsub_rn(sl[SX + ja], sl[SX + ia]), sl[SX + ia]);
  float Eay = __fmaf_rn(la, __fsub_rn(sl[SY + ja], sl[SY + ia]), sl[SY + ia]);
  float Ebx = __fmaf_rn(lb, __fsub_rn(sl[SX + jb], sl[SX + ib]), sl[SX + ib]);
  float Eby = __fmaf_rn(lb, __fsub_rn(sl[SY + jb], sl[SY + ib]), sl[SY + ib]);
  // E0 is the crossed edge with the smaller (lower, higher) global index key
  const int gua = min(g_l, g_a), gva = max(g_l, g_a);
  const int gub = min(g_l, g_b), gvb = max(g_l, g_b);
  bool swap = gub < gua || (gub == gua && gvb < gva);
  float E0x = swap ? Ebx : Eax, E0y = swap ? Eby : Eay;
  float E1x = swap ? Eax : Ebx, E1y = swap ? Eay : Eby;
  // |E32 - E64| per component; edge (lone, oa) is opposite ob and vice versa
  const float dE = fmaxf(sl[SDE + ob], sl[SDE + oa]);
  if (!(dE < 1e30f)) return 2;
  float e0 = __fmaf_rn(E0x, E0x, __fmul_rn(E0y, E0y));
  float e1 = __fmaf_rn(E1x, E1x, __fmul_rn(E1y, E1y));
  const float A0 = fabsf(E0x) + fabsf(E0y) + 2.0f * dE;  // bounds |E0x*| + |E0y*|
  const float A1 = fabsf(E1x) + fabsf(E1y) + 2.0f * dE;
  const float de0 = kSafety * (2.0f * A0 * dE + 3.01f * kU * e0) + 1e-37f;
  const float de1 = kSafety * (2.0f * A1 * dE + 3.01f * kU * e1) + 1e-37f;
  int c0 = count_estimate_f(e0, N, scale), c1 = count_estimate_f(e1, N, scale);
  // the two columns around each transition must be decided with certainty (this also rejects a
  // wrong estimate: one of the two differences is then <= 0)
  if (c0 > 0 && e0 - a2f[c0 - 1] <= de0 + kU * a2f[c0 - 1]) return 2;
  if (c0 < N && a2f[c0] - e0 <= de0 + kU * a2f[c0]) return 2;
  if (c1 > 0 && e1 - a2f[c1 - 1] <= de1 + kU * a2f[c1 - 1]) return 2;
  if (c1 < N && a2f[c1] - e1 <= de1 + kU * a2f[c1]) return 2;
  lo = min(c0, c1);
  hi = max(c0, c1);
  dlo = lo;
  if (lo > 0) {
    float Dx = __fsub_rn(E1x, E0x), Dy = __fsub_rn(E1y, E0y);
    const float dD = 2.0f * dE + kU * (fabsf(Dx) + fabsf(Dy));
    const float B = fabsf(Dx) + fabsf(Dy) + 2.0f * dD;  // bounds |Dx*| + |Dy*|
    // is the line's closest point C strictly inside the segment (E0.D < 0 < E1.D)?
    float d0 = __fmaf_rn(E0x, Dx, __fmul_rn(E0y, Dy));
    float d1 = __fmaf_rn(E1x, Dx, __fmul_rn(E1y, Dy));
    const float dd0 = kSafety * (A0 * dD + B * dE + 2.0f * kU * A0 * B) + 1e-37f;
    const float dd1 = kSafety * (A1 * dD + B * dE + 2.0f * kU * A1 * B) + 1e-37f;
    if (fabsf(d0) <= dd0 || fabsf(d1) <= dd1) return 2;
    if (d0 < 0.0f && d1 > 0.0f) {
      // alpha_c^2 |D|^2 > (E0 x D)^2  <=>  alpha_c^2 > h^2, h = |C| the segment's distance to
      // the axis.  C is inside the segment for the FP32 and the FP64 endpoints, and moving
      // each endpoint by at most dE per component moves h by at most sqrt(2) dE, so h^2 is
      // known to 2 h dh + dh^2 plus the rounding of the cross product, |D|^2 and the quotient.
      float cr = __fmaf_rn(E0x, Dy, -__fmul_rn(E0y, Dx));
      float dd = __fmaf_rn(Dx, Dx, __fmul_rn(Dy, Dy));
      if (!(dd >= 1e-30f && dd <= 1e30f)) return 2;  // keep the fast quotient in its range
      // fast quotient (at most 2 ulp = 4 kU relative from the rounded operands) and fast root
      // (used in the bound only, raised by 1e-6 relative to cover its own error)
      float h2 = __fdividef(__fmul_rn(cr, cr), dd);
      const float h = h2 > 0.0f ? h2 * rsqrtf(h2) * 1.000001f : 0.0f;
      const float dh = 1.5f * (dE + kU * B);
      const float rb = B * rsqrtf(dd);  // (|Dx| + |Dy| + 2 dD) / |D|
      const float dq = kSafety * (2.0f * h * dh + 2.0f * dh * dh + 4.0f * kU * h * A0 * rb +
                                  2.0f * kU * h2 * (1.0f + rb * rb) + 4.0f * kU * h2) + 1e-37f;
      if (!(dq < 1e30f)) return 2;
      const int cs = count_estimate_f(h2, N, scale);  // first column with alpha^2 > h^2
      if (cs >= lo) {
        if (h2 - a2f[lo - 1] <= dq + kU * a2f[lo - 1]) return 2;
      } else {
        if (cs > 0 && h2 - a2f[cs - 1] <= dq + kU * a2f[cs - 1]) return 2;
        if (a2f[cs] - h2 <= dq + kU * a2f[cs]) return 2;
        dlo = cs;
      }
    }
  }
  return 1;
}

__device__ __forceinline__ void add_intervals(int *row, int N, int lo, int hi, int dlo) {
  if (lo < hi) {
    atomicAdd(row + lo, 1);
    if (hi < N) atomicAdd(row + hi, -1);
  }
  if (dlo < lo) {
    atomicAdd(row + dlo, 2);
    if (lo < N) atomicAdd(row + lo, -2);
  }
}

// Candidate ranges of the grid cells around an oriented point, for every thread of the block:
// the (2 nhalf + 1)^3 cells around the spin vertex's cell (cell edge > reach / nhalf).  A
// triangle binned in a cell (by its bounding-sphere centre, radius <= r_big) can reach the
// support volume only if the cell's box lies within `reach` of the spin vertex and the box's
// bounding sphere lies within r_big of the support cylinder (axis along the normal); other
// cells are skipped, and cells that hash to an already listed bucket are listed once.  On
// return entry i <= nneigh (the last one is the scene's big list) holds the candidate range
// [buckets[i], bdup[i]) (empty for skipped entries).  Ends with a block barrier.
__device__ __forceinline__ void neighbour_ranges(const KArgs &a, int64_t bucket_off,
                                                 uint32_t nbuckets, float Sx, float Sy, float Sz,
                                                 float nxf, float nyf, float nzf, int *buckets,
                                                 int *bdup, int tid, int nthreads) {
  const int nw_ = 2 * a.nhalf + 1, nneigh = nw_ * nw_ * nw_;
  float ux = 0.0f, uy = 0.0f, uz = 1.0f;  // axis direction (identity rule for a zero normal)
  {
    const float n2 = nxf * nxf + nyf * nyf + nzf * nzf;
    if (n2 > 1e-30f) {
      const float inv = rsqrtf(n2);
      ux = nxf * inv;
      uy = nyf * inv;
      uz = nzf * inv;
    }
  }
  for (int cidx = tid; cidx < nneigh; cidx += nthreads) {
    const int ix = cell_coord(Sx, a.inv_cell) + cidx % nw_ - a.nhalf;
    const int iy = cell_coord(Sy, a.inv_cell) + (cidx / nw_) % nw_ - a.nhalf;
    const int iz = cell_coord(Sz, a.inv_cell) + cidx / (nw_ * nw_) - a.nhalf;
    const float c = a.cell;
    const float gx = fmaxf(fmaxf((float)ix * c - Sx, Sx - (float)(ix + 1) * c), 0.0f);
    const float gy = fmaxf(fmaxf((float)iy * c - Sy, Sy - (float)(iy + 1) * c), 0.0f);
    const float gz = fmaxf(fmaxf((float)iz * c - Sz, Sz - (float)(iz + 1) * c), 0.0f);
    // box centre relative to the spin vertex, its axial and radial distances to the axis
    const float hb = 0.8660254f * c * 1.001f + 1e-3f * c;  // half diagonal (+ cell rounding)
    const float cx = ((float)ix + 0.5f) * c - Sx, cy = ((float)iy + 0.5f) * c - Sy,
                cz = ((float)iz + 0.5f) * c - Sz;
    const float ax = fabsf(cx * ux + cy * uy + cz * uz);
    const float rad2 = cx * cx + cy * cy + cz * cz - ax * ax;
    const float marg = hb + a.r_big + 1e-3f * a.reach + 1e-5f * (fabsf(cx) + fabsf(cy) + fabsf(cz));
    const float rl = a.alpha_cull + marg;
    const bool near = gx * gx + gy * gy + gz * gz <= a.reach * a.reach &&
                      ax <= a.beta_cull + marg && rad2 <= rl * rl;
    buckets[cidx] = near ? (int)(bucket_off + cell_hash(ix, iy, iz, nbuckets - 1)) : -1;
  }
  if (tid == 0) buckets[nneigh] = (int)(bucket_off + nbuckets);  // the scene's big list
  __syncthreads();
  for (int cidx = tid; cidx < nneigh; cidx += nthreads) {
    const int b = buckets[cidx];
    bool dup = b < 0;
    for (int k = 0; k < cidx && !dup; ++k) dup = buckets[k] == b;
    bdup[cidx] = dup ? 1 : 0;
  }
  if (tid == 0) bdup[nneigh] = 0;
  __syncthreads();
  // candidate range of every listed bucket, fetched once per block
  for (int cidx = tid; cidx <= nneigh; cidx += nthreads) {
    int beg = 0, end = 0;
    if (!bdup[cidx]) {
      const int b = buckets[cidx];
      beg = a.starts[b];
      end = a.starts[b + 1];
    }
    buckets[cidx] = beg;
    bdup[cidx] = end;
  }
  __syncthreads();
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 4 ? 7 : 3) k_generate(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t o = blockIdx.x;

  Shared s;
  {
    unsigned char *p = smem;
    s.diff = reinterpret_cast<int *>(p);
    p += ((size_t)N * N * 4 + 15) & ~(size_t)15;
    s.a2d = reinterpret_cast<double *>(p);
    s.bd = s.a2d + N;
    s.fr = s.bd + N;
    s.a2f = reinterpret_cast<float *>(s.fr + 8);
    s.bf = s.a2f + N;
    s.buckets = reinterpret_cast<int *>(s.bf + N);
    const int nn = (2 * a.nhalf + 1) * (2 * a.nhalf + 1) * (2 * a.nhalf + 1);
    s.bdup = s.buckets + nn + 1;
    int *wbase = s.bdup + nn + 1;
    s.wq = wbase + warp * kPerWarp;
    s.wst = s.wq;
    s.bq_rec = s.wq + 64;
    s.bq_r = reinterpret_cast<unsigned char *>(s.bq_rec + 64);
    s.slots = reinterpret_cast<float *>(s.bq_rec + 64 + 16);
  }

  const int64_t og = a.origin_base + o;  // launch-wide origin index
  const GenScene &sc = a.tab[scene_of_origin(a.tab, a.num_scenes, og)];
  const int64_t ol = og - sc.origin_off;  // origin index within its scene
  const int vid = sc.origins[ol];
  if (vid < 0 || vid >= sc.nv) {
    if (tid == 0) set_status(a.status, RICI_ERR_INDEX_OUT_OF_RANGE);
    return;
  }
  const float Sx = sc.V[3 * (int64_t)vid], Sy = sc.V[3 * (int64_t)vid + 1],
              Sz = sc.V[3 * (int64_t)vid + 2];
  const float nxf = sc.Nrm[3 * (int64_t)vid], nyf = sc.Nrm[3 * (int64_t)vid + 1],
              nzf = sc.Nrm[3 * (int64_t)vid + 2];
  const int64_t bucket_off = sc.bucket_off;
  const uint32_t nbuckets = sc.nbuckets;
  uint16_t *const out_img = sc.out + ol * (int64_t)N * N;
  if (!(isfinite(Sx) && isfinite(Sy) && isfinite(Sz) && isfinite(nxf) && isfinite(nyf) &&
        isfinite(nzf))) {
    if (tid == 0) set_status(a.status, RICI_ERR_NONFINITE_INPUT);
    return;
  }

  for (int i = tid; i < N * N; i += NW * 32) s.diff[i] = 0;
  const double Rd = (double)a.R;
  for (int i = tid; i < N; i += NW * 32) {
    double al = __ddiv_rn(__dmul_rn(Rd, (double)(2 * i + 1)), (double)(2 * N));
    double a2 = __dmul_rn(al, al);
    double b = __ddiv_rn(__dmul_rn(Rd, (double)(2 * i + 1 - N)), (double)(2 * N));
    s.a2d[i] = a2;
    s.bd[i] = b;
    s.a2f[i] = __double2float_rn(a2);
    s.bf[i] = __double2float_rn(b);
  }
  if (tid == 0) {
    s.fr[0] = Sx;
    s.fr[1] = Sy;
    s.fr[2] = Sz;
    frame_fp64(nxf, nyf, nzf, s.fr + 3);
  }
  __syncthreads();

  const float fax = __double2float_rn(s.fr[3]), fay = __double2float_rn(s.fr[4]);
  const float fbx = __double2float_rn(s.fr[5]), fbz = __double2float_rn(s.fr[6]);
  const float wx = fbx * fax, wy = fbx * fay, wz = fbz;  // central axis in world coordinates
  const float R = a.R;
  const float scale = (float)(2 * N) / R;
  const float spacing = R / (float)N;
  const float acull_xy = sqrtf(s.a2f[N - 1]) * (1.0f + 1.0f / 4096.0f);
  const bool fp64_only = a.mode == RICI_GEN_FP64;

  unsigned long long n_tri = 0, n_items = 0, n_band = 0, n_cand = 0;
  int qn = 0;  // warp-uniform candidate queue length
  int bn = 0;  // warp-uniform FP64 queue length

  // FP64 re-evaluation of queued band items, one per lane
  auto flush_band = [&](int cnt) {
    if (lane < cnt) {
      int lo = 0, hi = 0, dlo = 0;
      const int r = s.bq_r[lane];
      if (layer_fp64(a.rec, a.rs, s.fr, s.bd, s.a2d, N, s.bq_rec[lane], r, lo, hi, dlo))
        add_intervals(s.diff + r * N, N, lo, hi, dlo);
    }
    __syncwarp();
    const int rest = bn - cnt;
    int mr = 0, mq = 0;
    if (lane < rest) {
      mr = s.bq_rec[cnt + lane];
      mq = s.bq_r[cnt + lane];
    }
    __syncwarp();
    if (lane < rest) {
      s.bq_rec[lane] = mr;
      s.bq_r[lane] = mq;
    }
    bn = rest;
    __syncwarp();
  };

  auto process_batch = [&](int cnt) {
    // ---- per-triangle setup: one survivor per lane
    int nlay = 0;
    float *sl = s.slots + lane * kSlot;
    if (lane < cnt) {
      const int rec = s.wq[lane];
      float4 r1 = a.rec[a.rs + rec], r2 = a.rec[2 * a.rs + rec], r3 = a.rec[3 * a.rs + rec];
      float P[9] = {r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w, r3.x};
      float tx[3], ty[3], tz[3], M = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        M = fmaxf(M, project_fp32(P[3 * k], P[3 * k + 1], P[3 * k + 2], Sx, Sy, Sz, fax, fay, fbx,
                                  fbz, tx[k], ty[k], tz[k]));
      // |T32 - T64| <= dT for every coordinate (first-order bound 7uM, 10uM with slack)
      const float dT = 10.0f * kU * M + 1e-37f;
      const float dside = kSafety * (dT + kU * R);
      float zmin = fminf(fminf(tz[0], tz[1]), tz[2]), zmax = fmaxf(fmaxf(tz[0], tz[1]), tz[2]);
      float xl = fminf(fminf(tx[0], tx[1]), tx[2]), xh = fmaxf(fmaxf(tx[0], tx[1]), tx[2]);
      float yl = fminf(fminf(ty[0], ty[1]), ty[2]), yh = fmaxf(fmaxf(ty[0], ty[1]), ty[2]);
      float gx = fmaxf(0.0f, fmaxf(xl, -xh)), gy = fmaxf(0.0f, fmaxf(yl, -yh));
      float lim = acull_xy + 2.0f * dT;
      bool keep = gx * gx + gy * gy <= lim * lim;
      // layers whose side decision is not certainly identical for all three vertices
      int r_lo = 0, r_hi = -1;
      if (keep) {
        float zl = zmin - dside, zh = zmax + dside;
        float fl = ceilf((zl * scale + (float)(N - 1)) * 0.5f);
        r_lo = fl <= 0.0f ? 0 : (fl >= (float)N ? N : (int)fl);
        while (r_lo > 0 && s.bf[r_lo - 1] > zl) --r_lo;
        while (r_lo < N && s.bf[r_lo] <= zl) ++r_lo;
        float fh = floorf((zh * scale + (float)(N - 1)) * 0.5f);
        r_hi = fh < 0.0f ? -1 : (fh >= (float)(N - 1) ? N - 1 : (int)fh);
        while (r_hi < N - 1 && s.bf[r_hi + 1] <= zh) ++r_hi;
        while (r_hi >= 0 && s.bf[r_hi] > zh) --r_hi;
        nlay = max(0, r_hi - r_lo + 1);
      }
      if (nlay > 0) {
        unsigned meta = (unsigned)r_lo;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          sl[SX + k] = tx[k];
          sl[SY + k] = ty[k];
          sl[SZ + k] = tz[k];
          // side band: the one layer a vertex could be ambiguous against
          float fr_ = rintf((tz[k] * scale + (float)(N - 1)) * 0.5f);
          int rk = fr_ <= 0.0f ? 0 : (fr_ >= (float)(N - 1) ? N - 1 : (int)fr_);
          unsigned band = kNoBand;
          for (int d = -1; d <= 1; ++d) {
            int rr = rk + d;
            if (rr >= 0 && rr < N && fabsf(tz[k] - s.bf[rr]) <= dside) band = (unsigned)rr;
          }
          meta |= band << (8 * (k + 1));
        }
        if (fp64_only || dside >= 0.25f * spacing) meta = (meta & ~0xff00u) | (kAllBand << 8);
        sl[SGID + 0] = r3.y;
        sl[SGID + 1] = r3.z;
        sl[SGID + 2] = r3.w;
        // per-edge bound on |E32 - E64| per component (edge k is opposite vertex k):
        // E = T_u + lambda (T_v - T_u); lambda = (beta - z_u) / (z_v - z_u)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int i = k == 0 ? 1 : 0, j = k == 2 ? 1 : 2;
          const float den = fabsf(tz[j] - tz[i]);
          const float eden = 2.0f * dT + kU * den;
          // lambda = (beta - z_i) * (1 / (z_j - z_i)): reciprocal and product each round once
          const float el = (kU * R + dT + kU * den + eden) / (den - eden) + 3.0f * kU;
          const float ext = fmaxf(fabsf(tx[j] - tx[i]), fabsf(ty[j] - ty[i]));
          const float mag = fmaxf(fmaxf(fabsf(tx[i]), fabsf(tx[j])), fmaxf(fabsf(ty[i]), fabsf(ty[j])));
          const float de = 1.1f * (3.0f * dT + kU * (ext + mag) + (ext + 2.0f * dT) * el);
          sl[SDE + k] = (den > eden && de < 1e30f) ? de : __int_as_float(0x7f800000);
          sl[SINV + k] = __frcp_rn(tz[j] - tz[i]);
        }
        sl[SMETA] = __uint_as_float(meta);
        sl[SREC] = __int_as_float(rec);
      }
    }
    // ---- distribute (triangle, layer) items over the lanes
    int incl = nlay;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int first = incl - nlay;  // this lane's triangle owns items [first, first + nlay)
    n_tri += nlay > 0;
    for (int base = 0; base < total; base += 32) {
      const int it = base + lane;
      const bool act = it < total;
      // owner of each item of this window: every triangle with items in the window marks the
      // first window position it owns (positions are distinct; the triangle holding position 0
      // always marks it), and an item belongs to the triangle of the last mark at or before it
      const int d = first - base;
      const bool mark = nlay > 0 && d < 32 && d + nlay > 0;
      const int pos = d > 0 ? d : 0;
      if (mark) s.wst[pos] = lane;
      const unsigned starts = __reduce_or_sync(0xffffffffu, mark ? 1u << pos : 0u);
      __syncwarp();
      const int q = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));  // bit 0 is always set
      const int owner = s.wst[q];
      const int ofirst = __shfl_sync(0xffffffffu, first, owner);
      int res = 0, r = 0, rec = 0, lo = 0, hi = 0, dlo = 0;
      if (act) {
        const float *ts = s.slots + owner * kSlot;
        const unsigned meta = __float_as_uint(ts[SMETA]);
        r = (int)(meta & 0xffu) + (it - ofirst);
        rec = __float_as_int(ts[SREC]);
        const unsigned b0 = (meta >> 8) & 0xffu;
        const bool band = b0 == kAllBand || r == (int)b0 || r == (int)((meta >> 16) & 0xffu) ||
                          r == (int)(meta >> 24);
        res = band ? 2 : layer_fp32(s.bf, s.a2f, N, ts, r, scale, lo, hi, dlo);
        ++n_items;
      }
      // items inside the error band wait in the FP64 queue (evaluated 32 at a time)
      const unsigned bal = __ballot_sync(0xffffffffu, res == 2);
      if (res == 2) {
        const int pos = bn + __popc(bal & ((1u << lane) - 1u));
        s.bq_rec[pos] = rec;
        s.bq_r[pos] = r;
        ++n_band;
      }
      bn += __popc(bal);
      if (res == 1) add_intervals(s.diff + r * N, N, lo, hi, dlo);
      __syncwarp();
      if (bn >= 32) flush_band(32);
    }
    __syncwarp();
  };

  // ---- candidate triangles: the records of this point's scene, culled by the bounding spheres of
  // their 1024-record groups, then of the 32-record chunks of passing groups, then one by one.  A
  // sphere containing the bounding spheres of its records fails its test only if every record
  // fails the record test: the record test widened by the sphere's radius, with a margin that
  // covers the record test's own and both tests' rounding.
  const float mpos = 4e-7f * (fabsf(Sx) + fabsf(Sy) + fabsf(Sz));
  auto sphere_pass = [&](const float4 c) -> bool {
    if (!(c.w < 1e30f)) return true;
    const float dx = c.x - Sx, dy = c.y - Sy, dz = c.z - Sz;
    const float z = fmaf(wx, dx, fmaf(wy, dy, wz * dz));
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float m = 2e-3f * R + 2e-5f * (fabsf(dx) + fabsf(dy) + fabsf(dz) + 2.0f * c.w) + mpos;
    const float al = a.alpha_cull + c.w + m;
    return fabsf(z) <= a.beta_cull + c.w + m && d2 - z * z <= al * al;
  };
  const int64_t rb = a.starts[bucket_off], re = a.starts[bucket_off + nbuckets + 1];
  if (re > rb) {
    const int64_t c_lo = rb >> kChunkShift, c_hi = (re - 1) >> kChunkShift;
    const int64_t g_lo = rb >> kGroupShift, ng = ((re - 1) >> kGroupShift) - g_lo + 1;
    // group g_lo + k0 + lane * NW + warp: consecutive groups (neighbours in space) go to
    // different warps
    for (int64_t k0 = 0; k0 < ng; k0 += 32 * NW) {
      const int64_t gi = k0 + (int64_t)lane * NW + warp;
      const bool gp = gi < ng && sphere_pass(a.grp[g_lo + gi]);
      unsigned gm = __ballot_sync(0xffffffffu, gp);
      while (gm) {
        const int64_t g = g_lo + k0 + (int64_t)(__ffs(gm) - 1) * NW + warp;
        gm &= gm - 1;
        const int64_t ci = (g << (kGroupShift - kChunkShift)) + lane;
        const bool cp = ci >= c_lo && ci <= c_hi && sphere_pass(a.chk[ci]);
        unsigned cm = __ballot_sync(0xffffffffu, cp);
        // records of the passing chunks; the next chunk's spheres are loaded before the current
        // ones are tested and queued, so the load's latency overlaps that work
        int64_t t = 0;
        float4 cn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        bool more = cm != 0;
        if (more) {
          t = (((g << (kGroupShift - kChunkShift)) + __ffs(cm) - 1) << kChunkShift) + lane;
          cm &= cm - 1;
          if (t >= rb && t < re) cn = a.rec[t];
        }
        while (more) {
          const int64_t tc = t;
          const float4 c = cn;
          more = cm != 0;
          if (more) {
            t = (((g << (kGroupShift - kChunkShift)) + __ffs(cm) - 1) << kChunkShift) + lane;
            cm &= cm - 1;
            if (t >= rb && t < re) cn = a.rec[t];
          }
          bool pass = false;
          if (tc >= rb && tc < re) {
            float dx = c.x - Sx, dy = c.y - Sy, dz = c.z - Sz;
            float z = fmaf(wx, dx, fmaf(wy, dy, wz * dz));
            float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float m = 1e-3f * R + 1e-5f * (fabsf(dx) + fabsf(dy) + fabsf(dz));
            float al = a.alpha_cull + c.w + m;
            pass = fabsf(z) <= a.beta_cull + c.w + m && d2 - z * z <= al * al;
            ++n_cand;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, pass);
          if (pass) s.wq[qn + __popc(bal & ((1u << lane) - 1u))] = (int)tc;
          qn += __popc(bal);
          __syncwarp();
          if (qn >= 32) {
            process_batch(32);
            int rest = qn - 32;
            int moved = lane < rest ? s.wq[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) s.wq[lane] = moved;
            qn = rest;
            __syncwarp();
          }
        }
      }
    }
  }
  if (qn > 0) process_batch(qn);
  if (bn > 0) flush_band(bn);

  if (a.counters) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      n_tri += __shfl_down_sync(0xffffffffu, n_tri, d);
      n_items += __shfl_down_sync(0xffffffffu, n_items, d);
      n_band += __shfl_down_sync(0xffffffffu, n_band, d);
      n_cand += __shfl_down_sync(0xffffffffu, n_cand, d);
    }
    if (lane == 0) {
      atomicAdd(a.counters + 0, n_tri);
      atomicAdd(a.counters + 1, n_items);
      atomicAdd(a.counters + 2, n_band);
      atomicAdd(a.counters + 3, n_cand);
    }
  }
  __syncthreads();

  // ---- prefix-sum each row of the difference image, saturate, store uint16
  uint16_t *out = out_img;
  const int cpl = (N + 31) / 32;
  if ((N == 64 || N == 128) && (reinterpret_cast<uintptr_t>(out) & 7) == 0) {
    // each lane owns 2 (N = 64) or 4 (N = 128) consecutive columns: one vector load of the
    // difference row and one 32- or 64-bit store of the packed counts
    for (int r = warp; r < N; r += NW) {
      const int *row = s.diff + r * N;
      int v0, v1, v2 = 0, v3 = 0;
      if (cpl == 2) {
        const int2 x = *reinterpret_cast<const int2 *>(row + 2 * lane);
        v0 = x.x;
        v1 = x.y;
      } else {
        const int4 x = *reinterpret_cast<const int4 *>(row + 4 * lane);
        v0 = x.x;
        v1 = x.y;
        v2 = x.z;
        v3 = x.w;
      }
      const int sum = v0 + v1 + v2 + v3;
      int incl = sum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const int p0 = incl - sum + v0, p1 = p0 + v1, p2 = p1 + v2, p3 = p2 + v3;
      const uint32_t w0 = (uint32_t)min(max(p0, 0), 65535) | ((uint32_t)min(max(p1, 0), 65535) << 16);
      if (cpl == 2) {
        *reinterpret_cast<uint32_t *>(out + r * N + 2 * lane) = w0;
      } else {
        const uint32_t w1 =
            (uint32_t)min(max(p2, 0), 65535) | ((uint32_t)min(max(p3, 0), 65535) << 16);
        *reinterpret_cast<uint2 *>(out + r * N + 4 * lane) = make_uint2(w0, w1);
      }
    }
    return;
  }
  for (int r = warp; r < N; r += NW) {
    const int *row = s.diff + r * N;
    const int c0 = lane * cpl, c1 = min(N, c0 + cpl);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += row[c];
    int incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    int run = incl - sum;
    for (int c = c0; c < c1; ++c) {
      run += row[c];
      out[r * N + c] = (uint16_t)min(max(run, 0), 65535);
    }
  }
}

size_t generate_smem_bytes(int N, int nhalf, int warps) {
  const int nn = (2 * nhalf + 1) * (2 * nhalf + 1) * (2 * nhalf + 1);
  size_t b = ((size_t)N * N * 4 + 15) & ~(size_t)15;
  b += (size_t)(2 * N + 8) * sizeof(double);
  b += (size_t)(2 * N) * sizeof(float);
  b += 2 * (size_t)(nn + 1) * sizeof(int);
  b += (size_t)warps * kPerWarp * 4;
  return b;
}

template <int NW>
cudaError_t launch_k_generate(const KArgs &k, int64_t total_origins, cudaStream_t st) {
  const size_t smem = generate_smem_bytes(k.N, k.nhalf, NW);
  cudaError_t e = cudaFuncSetAttribute(k_generate<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  for (int64_t o0 = 0; o0 < total_origins; o0 += 0x7fffffff) {
    const int64_t cnt = total_origins - o0 < 0x7fffffff ? total_origins - o0 : 0x7fffffff;
    KArgs kk = k;
    kk.origin_base = o0;
    k_generate<NW><<<(unsigned)cnt, NW * 32, smem, st>>>(kk);
    count_launches(1);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ clutter measure
// Eq. clutter (Section 4.1): clutter = (A_all - A_object) / A_all with A_all the surface area
// inside the support volume of an oriented point and A_object the part on the object of
// interest.  The support volume is the image's cylinder: Tx^2 + Ty^2 <= R^2, |Tz| <= R/2 in the
// frame of Eqs. relativeLocation..secondRotation (a rotation, so frame areas are scene areas).

// Signed area of the triangle (0, p, q) that lies inside the disk |x| <= R (R2 = R^2), in the
// (Tx, Ty) plane.  The segment p-q is inside the disk for t in [t1, t2] (roots of
// |p + t (q - p)|^2 = R^2) and outside elsewhere; clipped to [0, 1] this gives three pieces: an
// outer piece adds the circular sector it subtends, the inner one the triangle with the origin.
__device__ double disk_wedge(double px, double py, double qx, double qy, double R2) {
  const double dx = qx - px, dy = qy - py;
  const double A = dx * dx + dy * dy;
  double ta = 1.0, tb = 1.0;  // no crossing: the whole segment is outside
  if (A > 0.0) {
    const double B = px * dx + py * dy, C = px * px + py * py - R2;
    const double disc = B * B - A * C;
    if (disc > 0.0) {
      const double sq = sqrt(disc);
      ta = fmin(fmax((-B - sq) / A, 0.0), 1.0);
      tb = fmin(fmax((-B + sq) / A, 0.0), 1.0);
    }
  }
  const double ax = px + ta * dx, ay = py + ta * dy, bx = px + tb * dx, by = py + tb * dy;
  // an outer piece never spans opposite directions (the segment between them would cross the
  // disk), so a zero cross product means an empty sector; this also keeps a zero-length piece
  // at the origin, whose dot product may be -0, from reading as an angle of pi
  const double c0 = px * ay - py * ax, c1 = bx * qy - by * qx;
  const double s0 = c0 == 0.0 ? 0.0 : atan2(c0, px * ax + py * ay);  // sector p .. P(ta)
  const double s1 = c1 == 0.0 ? 0.0 : atan2(c1, bx * qx + by * qy);  // sector P(tb) .. q
  return 0.5 * R2 * (s0 + s1) + 0.5 * (ax * by - ay * bx);
}

// Area of the part of one projected triangle inside the support volume: clip it to the slab
// |Tz| <= R/2, then area(projection onto (Tx, Ty) within the disk) / |cos|, cos the z component
// of the unit normal.  Planes with |cos| < 1e-7 count as parallel to the axis: the polygon is cut
// by the two lines where the plane, at its mean distance p from the axis, meets the cylinder
// (|h| <= sqrt(R^2 - p^2), h the horizontal in-plane coordinate).
__device__ double support_area64(const double T[3][3], double R) {
  const double ux = T[1][0] - T[0][0], uy = T[1][1] - T[0][1], uz = T[1][2] - T[0][2];
  const double vx = T[2][0] - T[0][0], vy = T[2][1] - T[0][1], vz = T[2][2] - T[0][2];
  const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
  const double nn = sqrt(nx * nx + ny * ny + nz * nz);
  if (nn == 0.0) return 0.0;
  const double H = 0.5 * R;
  // the volume is convex: a triangle whose vertices all lie in it lies in it whole
  bool whole = true;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    whole = whole && T[i][0] * T[i][0] + T[i][1] * T[i][1] <= R * R && fabs(T[i][2]) <= H;
  if (whole) return 0.5 * nn;
  // slab clip (z <= H, then -z <= H), at most 5 vertices
  double P[5][3], Q[5][3];
  int m = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = i == 2 ? 0 : i + 1;
    const double di = H - T[i][2], dj = H - T[j][2];
    if (di >= 0.0) {
      P[m][0] = T[i][0]; P[m][1] = T[i][1]; P[m][2] = T[i][2];
      ++m;
    }
    if ((di >= 0.0) != (dj >= 0.0)) {
      const double f = di / (di - dj);
      P[m][0] = T[i][0] + f * (T[j][0] - T[i][0]);
      P[m][1] = T[i][1] + f * (T[j][1] - T[i][1]);
      P[m][2] = T[i][2] + f * (T[j][2] - T[i][2]);
      ++m;
    }
  }
  if (m < 3) return 0.0;
  int k = 0;
  for (int i = 0; i < m; ++i) {
    const int j = i + 1 == m ? 0 : i + 1;
    const double di = H + P[i][2], dj = H + P[j][2];
    if (di >= 0.0) {
      Q[k][0] = P[i][0]; Q[k][1] = P[i][1]; Q[k][2] = P[i][2];
      ++k;
    }
    if ((di >= 0.0) != (dj >= 0.0)) {
      const double f = di / (di - dj);
      Q[k][0] = P[i][0] + f * (P[j][0] - P[i][0]);
      Q[k][1] = P[i][1] + f * (P[j][1] - P[i][1]);
      Q[k][2] = P[i][2] + f * (P[j][2] - P[i][2]);
      ++k;
    }
  }
  if (k < 3) return 0.0;
  const double cz = fabs(nz) / nn;
  if (cz >= 1e-7) {
    double a = 0.0;
    for (int i = 0; i < k; ++i) {
      const int j = i + 1 == k ? 0 : i + 1;
      a += disk_wedge(Q[i][0], Q[i][1], Q[j][0], Q[j][1], R * R);
    }
    return fabs(a) / cz;
  }
  // plane parallel to the axis: in-plane coordinates (h, z), h along (-ny, nx) / |n_xy|
  const double hxy = sqrt(nx * nx + ny * ny);
  const double ex = -ny / hxy, ey = nx / hxy;
  double p = 0.0;
  for (int i = 0; i < k; ++i) p += (Q[i][0] * nx + Q[i][1] * ny) / hxy;
  p /= (double)k;
  if (fabs(p) >= R) return 0.0;
  const double c = sqrt(R * R - p * p);
  // area of the polygon's part with |h| <= c: shoelace over the polygon clipped to the band
  double G[7][2], E[7][2];
  for (int i = 0; i < k; ++i) {
    G[i][0] = Q[i][0] * ex + Q[i][1] * ey;
    G[i][1] = Q[i][2];
  }
  int g = k;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const double sg = side == 0 ? 1.0 : -1.0;
    int e = 0;
    for (int i = 0; i < g; ++i) {
      const int j = i + 1 == g ? 0 : i + 1;
      const double di = c - sg * G[i][0], dj = c - sg * G[j][0];
      if (di >= 0.0) {
        E[e][0] = G[i][0]; E[e][1] = G[i][1];
        ++e;
      }
      if ((di >= 0.0) != (dj >= 0.0)) {
        const double f = di / (di - dj);
        E[e][0] = G[i][0] + f * (G[j][0] - G[i][0]);
        E[e][1] = G[i][1] + f * (G[j][1] - G[i][1]);
        ++e;
      }
    }
    for (int i = 0; i < e; ++i) {
      G[i][0] = E[i][0];
      G[i][1] = E[i][1];
    }
    g = e;
  }
  if (g < 3) return 0.0;
  double a = 0.0;
  for (int i = 0; i < g; ++i) {
    const int j = i + 1 == g ? 0 : i + 1;
    a += G[i][0] * G[j][1] - G[j][0] * G[i][1];
  }
  return 0.5 * fabs(a);
}

constexpr int kClutterWarps = 4;
constexpr int kClutterMaxCells = 7 * 7 * 7 + 1;  // neighbourhoods of nhalf <= 3, + the big list

// One block per oriented point: the candidates of the neighbouring cells pass the same
// sphere-against-cylinder pretest as generation (limits of the full cylinder), queue per warp,
// and are evaluated 32 at a time in FP64, one per lane.  A triangle belongs to the object when
// its first vertex index is below object_vertices.
__global__ void __launch_bounds__(kClutterWarps * 32, 5)
    k_clutter(KArgs a, int64_t object_vertices, double *__restrict__ out_all,
              double *__restrict__ out_obj, double *__restrict__ out_clutter) {
  __shared__ int buckets[kClutterMaxCells], bdup[kClutterMaxCells];
  __shared__ double fr[7];
  __shared__ int wq[kClutterWarps][64];
  __shared__ double cq[kClutterWarps][64][9];  // projected triangles waiting to be clipped
  __shared__ unsigned char cq_obj[kClutterWarps][64];
  __shared__ double part[kClutterWarps][2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t og = a.origin_base + blockIdx.x;
  const GenScene &sc = a.tab[scene_of_origin(a.tab, a.num_scenes, og)];
  const int vid = sc.origins[og - sc.origin_off];
  if (vid < 0 || vid >= sc.nv) {
    if (tid == 0) {
      set_status(a.status, RICI_ERR_INDEX_OUT_OF_RANGE);
      out_all[og] = out_obj[og] = nan("");
      if (out_clutter) out_clutter[og] = nan("");
    }
    return;
  }
  const float Sx = sc.V[3 * (int64_t)vid], Sy = sc.V[3 * (int64_t)vid + 1],
              Sz = sc.V[3 * (int64_t)vid + 2];
  const float nxf = sc.Nrm[3 * (int64_t)vid], nyf = sc.Nrm[3 * (int64_t)vid + 1],
              nzf = sc.Nrm[3 * (int64_t)vid + 2];
  if (!(isfinite(Sx) && isfinite(Sy) && isfinite(Sz) && isfinite(nxf) && isfinite(nyf) &&
        isfinite(nzf))) {
    if (tid == 0) {
      set_status(a.status, RICI_ERR_NONFINITE_INPUT);
      out_all[og] = out_obj[og] = nan("");
      if (out_clutter) out_clutter[og] = nan("");
    }
    return;
  }
  if (tid == 0) {
    fr[0] = Sx;
    fr[1] = Sy;
    fr[2] = Sz;
    frame_fp64(nxf, nyf, nzf, fr + 3);
  }
  neighbour_ranges(a, sc.bucket_off, sc.nbuckets, Sx, Sy, Sz, nxf, nyf, nzf, buckets, bdup, tid,
                   kClutterWarps * 32);
  const float fax = __double2float_rn(fr[3]), fay = __double2float_rn(fr[4]);
  const float fbx = __double2float_rn(fr[5]), fbz = __double2float_rn(fr[6]);
  const float wx = fbx * fax, wy = fbx * fay, wz = fbz;  // central axis in world coordinates
  const double R = a.R;
  double acc_all = 0.0, acc_obj = 0.0;
  int qn = 0;  // warp-uniform candidate queue length
  int cn = 0;  // warp-uniform clip queue length
  // triangles that cross the volume's boundary, 32 at a time, so that a warp's lanes all take
  // the clipping path together
  auto clip_batch = [&](int cnt) {
    if (lane < cnt) {
      double T[3][3];
#pragma unroll
      for (int i = 0; i < 9; ++i) T[i / 3][i % 3] = cq[warp][lane][i];
      const double ar = support_area64(T, R);
      acc_all += ar;
      if (cq_obj[warp][lane]) acc_obj += ar;
    }
    __syncwarp();
  };
  // projected survivors: a triangle with its three vertices in the (convex) volume adds its
  // whole area at once; the others queue for clipping
  auto process = [&](int cnt) {
    bool clip = false, obj = false;
    double T[3][3];
    if (lane < cnt) {
      const int64_t r = wq[warp][lane];
      const float4 r1 = a.rec[a.rs + r], r2 = a.rec[2 * a.rs + r], r3 = a.rec[3 * a.rs + r];
      project64(r1.x, r1.y, r1.z, fr, T[0]);
      project64(r1.w, r2.x, r2.y, fr, T[1]);
      project64(r2.z, r2.w, r3.x, fr, T[2]);
      obj = __float_as_int(r3.y) < object_vertices;
      bool whole = true;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        whole = whole && T[i][0] * T[i][0] + T[i][1] * T[i][1] <= R * R &&
                fabs(T[i][2]) <= 0.5 * R;
      if (whole) {
        const double ux = T[1][0] - T[0][0], uy = T[1][1] - T[0][1], uz = T[1][2] - T[0][2];
        const double vx = T[2][0] - T[0][0], vy = T[2][1] - T[0][1], vz = T[2][2] - T[0][2];
        const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        const double ar = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
        acc_all += ar;
        if (obj) acc_obj += ar;
      } else {
        clip = true;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, clip);
    if (clip) {
      const int pos = cn + __popc(bal & ((1u << lane) - 1u));
#pragma unroll
      for (int i = 0; i < 9; ++i) cq[warp][pos][i] = T[i / 3][i % 3];
      cq_obj[warp][pos] = obj ? 1 : 0;
    }
    cn += __popc(bal);
    __syncwarp();
    if (cn >= 32) {
      clip_batch(32);
      const int rest = cn - 32;  // entries 32.. move down to 0.. (sources and targets disjoint)
      if (lane < rest) {
#pragma unroll
        for (int i = 0; i < 9; ++i) cq[warp][lane][i] = cq[warp][32 + lane][i];
        cq_obj[warp][lane] = cq_obj[warp][32 + lane];
      }
      cn = rest;
      __syncwarp();
    }
  };
  const int nneigh = (2 * a.nhalf + 1) * (2 * a.nhalf + 1) * (2 * a.nhalf + 1);
  for (int nb = 0; nb <= nneigh; ++nb) {
    const int64_t beg = buckets[nb], end = bdup[nb];
    for (int64_t base = beg + warp * 32; base < end; base += kClutterWarps * 32) {
      const int64_t t = base + lane;
      bool pass = false;
      if (t < end) {
        const float4 c = a.rec[t];
        const float dx = c.x - Sx, dy = c.y - Sy, dz = c.z - Sz;
        const float z = fmaf(wx, dx, fmaf(wy, dy, wz * dz));
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float mg = 1e-3f * a.R + 1e-5f * (fabsf(dx) + fabsf(dy) + fabsf(dz));
        const float al = a.alpha_cull + c.w + mg;
        pass = fabsf(z) <= a.beta_cull + c.w + mg && d2 - z * z <= al * al;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, pass);
      if (pass) wq[warp][qn + __popc(bal & ((1u << lane) - 1u))] = (int)t;
      qn += __popc(bal);
      __syncwarp();
      if (qn >= 32) {
        process(32);
        const int rest = qn - 32;
        const int moved = lane < rest ? wq[warp][32 + lane] : 0;
        __syncwarp();
        if (lane < rest) wq[warp][lane] = moved;
        qn = rest;
        __syncwarp();
      }
    }
  }
  if (qn > 0) process(qn);
  if (cn > 0) clip_batch(cn);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    acc_all += __shfl_down_sync(0xffffffffu, acc_all, d);
    acc_obj += __shfl_down_sync(0xffffffffu, acc_obj, d);
  }
  if (lane == 0) {
    part[warp][0] = acc_all;
    part[warp][1] = acc_obj;
  }
  __syncthreads();
  if (tid == 0) {
    double sa = 0.0, so = 0.0;
    for (int w = 0; w < kClutterWarps; ++w) {
      sa += part[w][0];
      so += part[w][1];
    }
    out_all[og] = sa;
    out_obj[og] = so;
    // Eq. clutter: the share of the area inside the support volume not on the object
    if (out_clutter) out_clutter[og] = sa > 0.0 ? __ddiv_rn(__dsub_rn(sa, so), sa) : nan("");
  }
}

// ------------------------------------------------------------------ spin images
// Spin images (Section 2.1) from point samples of the mesh, with the FP32 projection stage of
// the generation kernel (Eqs. relativeLocation..secondRotation, frame rounded from FP64).
// Samples: m^2 per triangle at the centroids of the m^2 congruent sub-triangles of a division of
// every side into m parts, P = A + a (B - A) + b (C - A) with barycentric (a, b) = ((3i+1)/3m,
// (3j+1)/3m) for the upward sub-triangles (i + j <= m - 1) and ((3i+2)/3m, (3j+2)/3m) for the
// downward ones (i + j <= m - 2).  The plane is R wide and R high with the spin vertex at half
// height, N x N bins centred at alpha_c = (c + 1/2) R/N and beta_r = (r + 1/2 - N/2) R/N; a
// sample with alpha^2 < R^2 and -R/2 <= beta < R/2 adds bilinear weights to the four bins around
// it (weight on a bin outside the image is dropped).  Weights are formed in FP32 with explicit
// roundings and summed exactly as integers in units of 2^-24 (w * 2^24 rounded to the nearest
// integer) in shared memory, so the sums do not depend on the order of the samples; the image
// stores float32(sum * 2^-24).
constexpr int kSpinWarps = 4;
constexpr int kSpinMaxSide = 16;  // samples per triangle <= 256

__global__ void __launch_bounds__(kSpinWarps * 32) k_spin(KArgs a, int m, float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char spin_smem[];
  __shared__ int buckets[kClutterMaxCells], bdup[kClutterMaxCells];
  __shared__ double fr[7];
  __shared__ float smp_a[kSpinMaxSide * kSpinMaxSide], smp_b[kSpinMaxSide * kSpinMaxSide];
  __shared__ int wq[kSpinWarps][64];
  const int N = a.N;
  unsigned long long *img = reinterpret_cast<unsigned long long *>(spin_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t og = a.origin_base + blockIdx.x;
  const GenScene &sc = a.tab[scene_of_origin(a.tab, a.num_scenes, og)];
  float *dst = out + og * (int64_t)N * N;
  const int vid = sc.origins[og - sc.origin_off];
  bool bad = vid < 0 || vid >= sc.nv;
  float Sx = 0.0f, Sy = 0.0f, Sz = 0.0f, nxf = 0.0f, nyf = 0.0f, nzf = 1.0f;
  if (!bad) {
    Sx = sc.V[3 * (int64_t)vid];
    Sy = sc.V[3 * (int64_t)vid + 1];
    Sz = sc.V[3 * (int64_t)vid + 2];
    nxf = sc.Nrm[3 * (int64_t)vid];
    nyf = sc.Nrm[3 * (int64_t)vid + 1];
    nzf = sc.Nrm[3 * (int64_t)vid + 2];
  }
  const bool nonfinite = !bad && !(isfinite(Sx) && isfinite(Sy) && isfinite(Sz) &&
                                   isfinite(nxf) && isfinite(nyf) && isfinite(nzf));
  if (bad || nonfinite) {
    if (tid == 0)
      set_status(a.status, bad ? RICI_ERR_INDEX_OUT_OF_RANGE : RICI_ERR_NONFINITE_INPUT);
    for (int i = tid; i < N * N; i += kSpinWarps * 32) dst[i] = 0.0f;
    return;
  }
  for (int i = tid; i < N * N; i += kSpinWarps * 32) img[i] = 0ull;
  if (tid == 0) {
    fr[0] = Sx;
    fr[1] = Sy;
    fr[2] = Sz;
    frame_fp64(nxf, nyf, nzf, fr + 3);
    // sample table: upward sub-triangles row by row, then the downward ones
    const float den = (float)(3 * m);
    int k = 0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; i + j <= m - 1; ++j, ++k) {
        smp_a[k] = __fdiv_rn((float)(3 * i + 1), den);
        smp_b[k] = __fdiv_rn((float)(3 * j + 1), den);
      }
    for (int i = 0; i + 1 < m; ++i)
      for (int j = 0; i + j <= m - 2; ++j, ++k) {
        smp_a[k] = __fdiv_rn((float)(3 * i + 2), den);
        smp_b[k] = __fdiv_rn((float)(3 * j + 2), den);
      }
  }
  neighbour_ranges(a, sc.bucket_off, sc.nbuckets, Sx, Sy, Sz, nxf, nyf, nzf, buckets, bdup, tid,
                   kSpinWarps * 32);
  const float fax = __double2float_rn(fr[3]), fay = __double2float_rn(fr[4]);
  const float fbx = __double2float_rn(fr[5]), fbz = __double2float_rn(fr[6]);
  const float wx = fbx * fax, wy = fbx * fay, wz = fbz;  // central axis in world coordinates
  const float R = a.R, R2 = __fmul_rn(R, R), H = __fmul_rn(0.5f, R);
  const float scale = __fdiv_rn((float)N, R);
  const int ns = m * m;
  int qn = 0;
  auto process = [&](int cnt) {
    if (lane < cnt) {
      const int64_t r = wq[warp][lane];
      const float4 r1 = a.rec[a.rs + r], r2 = a.rec[2 * a.rs + r], r3 = a.rec[3 * a.rs + r];
      const float A[3] = {r1.x, r1.y, r1.z}, B[3] = {r1.w, r2.x, r2.y}, C[3] = {r2.z, r2.w, r3.x};
      const float ba[3] = {__fsub_rn(B[0], A[0]), __fsub_rn(B[1], A[1]), __fsub_rn(B[2], A[2])};
      const float ca[3] = {__fsub_rn(C[0], A[0]), __fsub_rn(C[1], A[1]), __fsub_rn(C[2], A[2])};
      for (int k = 0; k < ns; ++k) {
        const float sa = smp_a[k], sb = smp_b[k];
        const float px = __fmaf_rn(sb, ca[0], __fmaf_rn(sa, ba[0], A[0]));
        const float py = __fmaf_rn(sb, ca[1], __fmaf_rn(sa, ba[1], A[1]));
        const float pz = __fmaf_rn(sb, ca[2], __fmaf_rn(sa, ba[2], A[2]));
        float tx, ty, tz;
        project_fp32(px, py, pz, Sx, Sy, Sz, fax, fay, fbx, fbz, tx, ty, tz);
        const float a2 = __fmaf_rn(tx, tx, __fmul_rn(ty, ty));
        if (!(a2 < R2) || !(tz >= -H) || !(tz < H)) continue;
        const float u = __fmaf_rn(__fsqrt_rn(a2), scale, -0.5f);
        const float v = __fmaf_rn(__fadd_rn(tz, H), scale, -0.5f);
        const float cu = floorf(u), rv = floorf(v);
        const float fu = __fsub_rn(u, cu), fv = __fsub_rn(v, rv);
        const float gu = __fsub_rn(1.0f, fu), gv = __fsub_rn(1.0f, fv);
        const int c = (int)cu, rr = (int)rv;
        const bool c0 = c >= 0, c1 = c + 1 < N, r0 = rr >= 0, r1_ = rr + 1 < N;
        constexpr float kUnit = 16777216.0f;  // 2^24 units per sample
        if (r0 && c0)
          atomicAdd(img + rr * N + c, __float2ull_rn(__fmul_rn(__fmul_rn(gu, gv), kUnit)));
        if (r0 && c1)
          atomicAdd(img + rr * N + c + 1, __float2ull_rn(__fmul_rn(__fmul_rn(fu, gv), kUnit)));
        if (r1_ && c0)
          atomicAdd(img + (rr + 1) * N + c, __float2ull_rn(__fmul_rn(__fmul_rn(gu, fv), kUnit)));
        if (r1_ && c1)
          atomicAdd(img + (rr + 1) * N + c + 1,
                    __float2ull_rn(__fmul_rn(__fmul_rn(fu, fv), kUnit)));
      }
    }
    __syncwarp();
  };
  const int nneigh = (2 * a.nhalf + 1) * (2 * a.nhalf + 1) * (2 * a.nhalf + 1);
  for (int nb = 0; nb <= nneigh; ++nb) {
    const int64_t beg = buckets[nb], end = bdup[nb];
    for (int64_t base = beg + warp * 32; base < end; base += kSpinWarps * 32) {
      const int64_t t = base + lane;
      bool pass = false;
      if (t < end) {
        const float4 c = a.rec[t];
        const float dx = c.x - Sx, dy = c.y - Sy, dz = c.z - Sz;
        const float z = fmaf(wx, dx, fmaf(wy, dy, wz * dz));
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float mg = 1e-3f * a.R + 1e-5f * (fabsf(dx) + fabsf(dy) + fabsf(dz));
        const float al = a.alpha_cull + c.w + mg;
        pass = fabsf(z) <= a.beta_cull + c.w + mg && d2 - z * z <= al * al;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, pass);
      if (pass) wq[warp][qn + __popc(bal & ((1u << lane) - 1u))] = (int)t;
      qn += __popc(bal);
      __syncwarp();
      if (qn >= 32) {
        process(32);
        const int rest = qn - 32;
        const int moved = lane < rest ? wq[warp][32 + lane] : 0;
        __syncwarp();
        if (lane < rest) wq[warp][lane] = moved;
        qn = rest;
        __syncwarp();
      }
    }
  }
  if (qn > 0) process(qn);
  __syncthreads();
  for (int i = tid; i < N * N; i += kSpinWarps * 32)
    dst[i] = __double2float_rn(__dmul_rn(__ull2double_rn(img[i]), 1.0 / 16777216.0));
}

}  // namespace

cudaError_t launch_project_fp32(const float *pts, int64_t n, const float *sv, const float *sn,
                                float *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  k_project_fp32<<<(unsigned)(want < 152 * 16 ? want : 152 * 16), 256, 0, st>>>(pts, n, sv, sn, out);
  count_launches(1);
  return cudaGetLastError();
}

// Bins every triangle of the scenes into the hashed grid for support volumes of radius amax and
// half-height bmax around each oriented point, and fills the grid fields of k (table, records,
// bucket starts, cell size, reach, pretest limits, neighbourhood width).
static cudaError_t bin_triangles(const GenScene *scenes, int num_scenes, int64_t nt, int64_t TB,
                                 double R, double amax, double bmax, void *ws, int *status,
                                 cudaStream_t st, KArgs &k, int max_cells_per_reach,
                                 bool morton) {
  Carver c(ws);
  GenScene *tab = c.take<GenScene>(num_scenes);
  int *counts = c.take<int>(TB);
  int *starts = c.take<int>(TB + 1);
  int *partials = c.take<int>(TB / kScanItems + 2);
  uint32_t *tb = c.take<uint32_t>(nt);
  int *ts = c.take<int>(nt);
  float4 *rec = c.take<float4>(4 * nt);
  int *bbox = c.take<int>(8 * (int64_t)num_scenes);
  float4 *chk = c.take<float4>((nt + 31) / 32);
  float4 *grp = c.take<float4>((nt + 1023) / 1024);

  cudaError_t e;
  for (int s0 = 0; s0 < num_scenes; s0 += kFillChunk) {
    GenFill f;
    f.n = num_scenes - s0 < kFillChunk ? num_scenes - s0 : kFillChunk;
    for (int i = 0; i < f.n; ++i) f.e[i] = scenes[s0 + i];
    k_fill_gen_table<<<1, 256, 0, st>>>(tab + s0, f, bbox + 8 * (int64_t)s0);
    count_launches(1);
  }

  // enclosing sphere radius of the support cylinder
  const double rho = sqrt(amax * amax + bmax * bmax) * (1.0 + 1.0 / 1024.0) + 1e-3 * R;
  const Tuning tu = current_tuning();
  GridParams gp;
  gp.r_big = (float)(tu.gen_big_radius * rho);
  // a triangle (centre c, radius <= r_big) reaching the support volume has |c - S| <= reach;
  // with cell > reach / nhalf its cell lies within +-nhalf cells of the spin vertex's cell
  const double reach = (rho + gp.r_big) * 1.001;
  const int cpr = tu.gen_cells_per_reach < max_cells_per_reach ? tu.gen_cells_per_reach
                                                               : max_cells_per_reach;
  const double cell = reach / cpr * 1.01;
  gp.inv_cell = (float)(1.0 / cell);
  gp.mask = 0;

  if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * TB, st)) != cudaSuccess) return e;
  const int tpb = 256;
  const int64_t want = (nt + tpb - 1) / tpb;
  const int grid = (int)(want < 152 * 32 ? (want > 0 ? want : 1) : 152 * 32);
  if (nt > 0) {
    if (morton) {
      k_tri_bbox<<<grid, tpb, 0, st>>>(tab, num_scenes, nt, bbox);
      count_launches(1);
    }
    k_tri_bin<<<grid, tpb, 0, st>>>(tab, num_scenes, nt, gp, morton ? bbox : nullptr, counts, tb,
                                    ts, status);
    count_launches(1);
  }
  const int nb = (int)((TB + kScanItems - 1) / kScanItems);
  k_scan_partials<<<nb, 256, 0, st>>>(counts, TB, partials);
  k_scan_top<<<1, 1024, 0, st>>>(partials, nb);
  k_scan_final<<<nb, 256, 0, st>>>(counts, TB, partials, starts);
  count_launches(3);
  if (nt > 0) {
    k_tri_scatter<<<grid, tpb, 0, st>>>(tab, num_scenes, nt, tb, ts, starts, rec);
    count_launches(1);
    if (morton) {
      k_chunk_spheres<<<(unsigned)((nt + 1023) / 1024), 1024, 0, st>>>(rec, starts + TB, chk, grp);
      count_launches(1);
    }
  }
  k.chk = chk;
  k.grp = grp;

  k.tab = tab;
  k.num_scenes = num_scenes;
  k.rec = rec;
  k.rs = nt;
  k.starts = starts;
  k.inv_cell = gp.inv_cell;
  k.cell = (float)cell;
  k.reach = (float)(reach + 1e-3 * cell);  // slack for the rounding of cell coordinates
  k.R = (float)R;
  k.alpha_cull = (float)(amax * (1.0 + 1.0 / 1024.0) + 1e-3 * R);
  k.beta_cull = (float)(bmax * (1.0 + 1.0 / 1024.0) + 1e-3 * R);
  k.nhalf = cpr;
  k.r_big = gp.r_big;
  k.status = status;
  return cudaSuccess;
}

cudaError_t launch_generate_batch(const GenScene *scenes, const GenerateBatch &g, void *ws,
                                  cudaStream_t st) {
  const int N = g.N;
  if (g.total_origins == 0) return cudaSuccess;
  // support cylinder: alpha <= alpha_{N-1}, |beta| <= beta_{N-1}
  const double R = g.R;
  const double amax = R * (2.0 * N - 1.0) / (2.0 * N);
  const double bmax = R * (N - 1.0) / (2.0 * N);
  KArgs k;
  cudaError_t e = bin_triangles(scenes, g.num_scenes, g.total_tris, g.total_buckets, R, amax,
                                bmax, ws, g.status, st, k, kGenMaxCellsPerReach, true);
  if (e != cudaSuccess) return e;
  k.nhalf = 0;  // no neighbour-cell list: candidates come from the sphere hierarchy
  k.R = g.R;
  k.N = N;
  k.mode = g.mode;
  k.counters = reinterpret_cast<unsigned long long *>(g.counters);
  const Tuning tu = current_tuning();
  return tu.gen_warps == 8 ? launch_k_generate<8>(k, g.total_origins, st)
                           : launch_k_generate<4>(k, g.total_origins, st);
}

cudaError_t launch_clutter(const ClutterArgs &a, void *ws, cudaStream_t st) {
  if (a.num_origins == 0) return cudaSuccess;
  GenScene sc = {};
  sc.V = a.vertices;
  sc.Nrm = a.normals;
  sc.tris = a.triangles;
  sc.origins = a.origins;
  sc.nv = a.num_vertices;
  sc.nt = a.num_triangles;
  sc.no = a.num_origins;
  sc.nbuckets = bucket_count(a.num_triangles);
  // the whole support cylinder: alpha <= R, |beta| <= R/2
  const double R = a.support_radius;
  KArgs k;
  cudaError_t e = bin_triangles(&sc, 1, a.num_triangles, (int64_t)sc.nbuckets + 1, R, R, 0.5 * R,
                                ws, a.status, st, k, kClutterMaxCellsPerReach, false);
  if (e != cudaSuccess) return e;
  k.N = 0;
  k.mode = 0;
  k.counters = nullptr;
  for (int64_t o0 = 0; o0 < a.num_origins; o0 += 0x7fffffff) {
    const int64_t cnt = a.num_origins - o0 < 0x7fffffff ? a.num_origins - o0 : 0x7fffffff;
    KArgs kk = k;
    kk.origin_base = o0;
    k_clutter<<<(unsigned)cnt, kClutterWarps * 32, 0, st>>>(kk, a.object_vertices, a.out_area_all,
                                                             a.out_area_object, a.out_clutter);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_spin(const SpinArgs &a, void *ws, cudaStream_t st) {
  if (a.num_origins == 0) return cudaSuccess;
  GenScene sc = {};
  sc.V = a.vertices;
  sc.Nrm = a.normals;
  sc.tris = a.triangles;
  sc.origins = a.origins;
  sc.nv = a.num_vertices;
  sc.nt = a.num_triangles;
  sc.no = a.num_origins;
  sc.nbuckets = bucket_count(a.num_triangles);
  // the support cylinder of the plane: alpha <= R, |beta| <= R/2
  const double R = a.support_radius;
  KArgs k;
  cudaError_t e = bin_triangles(&sc, 1, a.num_triangles, (int64_t)sc.nbuckets + 1, R, R, 0.5 * R,
                                ws, a.status, st, k, kClutterMaxCellsPerReach, false);
  if (e != cudaSuccess) return e;
  k.N = a.resolution;
  k.mode = 0;
  k.counters = nullptr;
  const size_t smem = sizeof(unsigned long long) * (size_t)a.resolution * a.resolution;
  if ((e = cudaFuncSetAttribute(k_spin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  for (int64_t o0 = 0; o0 < a.num_origins; o0 += 0x7fffffff) {
    const int64_t cnt = a.num_origins - o0 < 0x7fffffff ? a.num_origins - o0 : 0x7fffffff;
    KArgs kk = k;
    kk.origin_base = o0;
    k_spin<<<(unsigned)cnt, kSpinWarps * 32, smem, st>>>(kk, a.samples_side, a.out_images);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_generate(const GenerateArgs &a, void *ws, cudaStream_t st) {
  GenScene sc = {};
  sc.V = a.vertices;
  sc.Nrm = a.normals;
  sc.tris = a.triangles;
  sc.origins = a.origins;
  sc.out = a.out_images;
  sc.nv = a.num_vertices;
  sc.nt = a.num_triangles;
  sc.no = a.num_origins;
  sc.nbuckets = bucket_count(a.num_triangles);
  GenerateBatch b;
  b.num_scenes = 1;
  b.total_tris = a.num_triangles;
  b.total_origins = a.num_origins;
  b.total_buckets = (int64_t)sc.nbuckets + 1;
  b.R = a.support_radius;
  b.N = a.resolution;
  b.mode = a.mode;
  b.counters = a.counters;
  b.status = a.status;
  return launch_generate_batch(&sc, b, ws, st);
}

}  // namespace rici
