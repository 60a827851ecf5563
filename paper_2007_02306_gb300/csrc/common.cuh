// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rici.h"

namespace rici {

// Generation launch arguments (all device pointers except sizes/scalars).
struct GenerateArgs {
  const float *vertices;
  const float *normals;
  int64_t num_vertices;
  const int32_t *triangles;
  int64_t num_triangles;
  const int32_t *origins;
  int64_t num_origins;
  float support_radius;
  int32_t resolution;
  uint16_t *out_images;
  int32_t mode;
  int64_t *counters;  // optional device int64[4]
  int *status;        // device status word
};

// Byte size of the generation workspace.
// Enqueue generation on `stream` using `ws` (>= generate_workspace_bytes, 256-aligned).
cudaError_t launch_generate(const GenerateArgs &a, void *ws, cudaStream_t stream);

// Clutter measure (Eq. clutter): per oriented point, the surface area inside its support volume
// and the part of it on the object's triangles (first vertex index < object_vertices), FP64.
struct ClutterArgs {
  const float *vertices;
  const float *normals;
  int64_t num_vertices;
  const int32_t *triangles;
  int64_t num_triangles;
  const int32_t *origins;
  int64_t num_origins;
  float support_radius;
  int64_t object_vertices;
  double *out_area_all;
  double *out_area_object;
  double *out_clutter;  // NULL, or (A_all - A_object) / A_all per oriented point
  int *status;  // device status word
};
// Enqueue the clutter measure on `stream` using `ws` (>= generate_workspace_bytes).
cudaError_t launch_clutter(const ClutterArgs &a, void *ws, cudaStream_t stream);

// Spin images (Section 2.1) from samples_side^2 point samples per triangle, float32 [O][N][N].
struct SpinArgs {
  const float *vertices;
  const float *normals;
  int64_t num_vertices;
  const int32_t *triangles;
  int64_t num_triangles;
  const int32_t *origins;
  int64_t num_origins;
  float support_radius;
  int32_t resolution;
  int32_t samples_side;
  float *out_images;
  int *status;  // device status word
};
// Enqueue spin-image generation on `stream` using `ws` (>= generate_workspace_bytes).
cudaError_t launch_spin(const SpinArgs &a, void *ws, cudaStream_t stream);

// One scene of a multi-scene generation launch (entry of the device scene table).
struct GenScene {
  const float *V;
  const float *Nrm;
  const int32_t *tris;
  const int32_t *origins;
  uint16_t *out;
  int64_t nv, nt, no;
  int64_t tri_off, origin_off, bucket_off;  // starts in the launch-wide index spaces
  uint32_t nbuckets;  // hashed buckets (power of two); bucket_off + nbuckets is the big list
  uint32_t pad_;
};

struct GenerateBatch {
  int num_scenes;
  int64_t total_tris, total_origins, total_buckets;
  float R;
  int N;
  int mode;
  int64_t *counters;
  int *status;
};

// scenes: host array with every offset filled; the table is written to the workspace by kernels
// (no host memory is referenced after the call returns).
cudaError_t launch_generate_batch(const GenScene *scenes, const GenerateBatch &b, void *ws,
                                  cudaStream_t stream);

struct SearchArgs {
  const uint16_t *needles;
  int64_t num_needles;
  const uint16_t *haystack;
  int64_t num_haystack;
  int32_t resolution;
  const int64_t *true_match;
  int32_t *out_rank;
  int64_t *out_true_distance;
  int32_t *out_top1;
  int64_t *out_distances;
  int32_t mode;
  int64_t *counters;  // optional device int64[4]
  int *status;
};

int64_t search_workspace_bytes(int64_t num_needles, int64_t num_haystack, int32_t resolution,
                               int32_t mode);
cudaError_t launch_search(const SearchArgs &a, void *ws, cudaStream_t stream);

// One scene of a multi-scene search (entry of the device scene table).  Needle i of the scene is
// launch-wide needle qoff + i; haystack image j is launch-wide image hoff + j; top-1 indices and
// true matches are scene-local.
struct SearchScene {
  const uint16_t *needles;
  const uint16_t *haystack;
  const int64_t *match;  // null: identity
  int32_t *rank;
  int64_t *dtrue;        // may be null
  int32_t *top1;         // may be null
  int64_t Q, H, qoff, hoff, tile_off;
  int32_t tiles_m, tiles_n;
};

// Launch shapes that do not change any result (set through rici_set_tuning; see RiciTuning).
struct Tuning {
  int gen_cells_per_reach;  // generation grid: cells per triangle reach (2 or 3)
  float gen_big_radius;     // triangles wider than this fraction of the support sphere are
                            // listed once per scene instead of being binned
  int gen_warps;            // warps per oriented point (4 or 8)
  int tc_group_m;           // tensor-core needle tiles swept together over the haystack
};
Tuning current_tuning();

struct SearchBatch {
  int num_scenes;
  int64_t Qtot, Htot, Hmax, tiles_total;
  int N;
  int mode;
  int64_t *counters;
  int *status;
};

// Tensor-core tiles of a scene (128 needles x 256 haystack images).
void search_tiles(int64_t Q, int64_t H, int32_t *tiles_m, int32_t *tiles_n);

// A tile of one scene: needle rows [qbeg + 128 m, ...), haystack columns [hbeg + 256 n, ...),
// valid for scene-local rows < Q and columns < H.
struct TcTile {
  int64_t m, n;          // tile coordinates within the scene
  int64_t qbeg, hbeg;    // scene offsets in the launch-wide needle / haystack arrays
  int64_t Q, H;
};

// Needle tiles are swept in groups of group_m over the scene's haystack tiles (L2 reuse).
__device__ __forceinline__ TcTile search_tile_of(const SearchScene *tab, int ns, int64_t t,
                                                int group_m) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {  // last scene whose first tile is <= t (empty scenes own no tile)
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].tile_off <= t) lo = mid; else hi = mid - 1;
  }
  const SearchScene &sc = tab[lo];
  const int64_t tl = t - sc.tile_off;
  const int tiles_m = sc.tiles_m, tiles_n = sc.tiles_n;
  const int64_t per_group = (int64_t)group_m * tiles_n;
  const int64_t g = tl / per_group;
  const int64_t r = tl - g * per_group;
  const int64_t gm = min((int64_t)group_m, (int64_t)tiles_m - g * group_m);
  TcTile tt;
  tt.n = r / gm;
  tt.m = g * group_m + r % gm;
  tt.qbeg = sc.qoff;
  tt.hbeg = sc.hoff;
  tt.Q = sc.Q;
  tt.H = sc.H;
  return tt;
}

int64_t search_batch_workspace_bytes(int num_scenes, int64_t Qtot, int64_t Htot, int N, int mode);
// scenes: host array with every offset filled (copied into the workspace by kernels).
cudaError_t launch_search_batch(const SearchScene *scenes, const SearchBatch &b, void *ws,
                                cudaStream_t stream, int64_t *out_distances);

// Tensor-core search (tc_search.cu): operand encoding + persistent tcgen05 GEMM with the rank /
// top-1 epilogue for narrow x narrow pairs of every scene.  Fills nwide/hwide and the wide
// lists/counts (launch-wide indices).
bool tc_supported(int N);
int64_t tc_workspace_bytes(int64_t Q, int64_t H, int N);
cudaError_t launch_tc_encode_and_rank(const SearchScene *tab, int num_scenes, const int *qscene,
                                      const int *hscene, int64_t Qtot, int64_t Htot,
                                      int64_t tiles_total, int N, void *ws, int *nwide, int *hwide,
                                      int *wn_list, int *wh_list, int *counts,
                                      const int *nflags, const int64_t *dtrue, int *rank,
                                      unsigned long long *best, int *status, int test_withhold,
                                      cudaStream_t st, const int *skip_needle = nullptr,
                                      const int *skip_tile = nullptr,
                                      const int *any_tile = nullptr);

// Integer tensor-core search (i8_search.cu): int8 operand encoding + mma.sync s8 GEMM with the
// rank / top-1 epilogue for int8-narrow x int8-narrow pairs of every scene (the tiles of the
// fp16 form).  Fills nwide/hwide (|delta| > 127) and the wide lists/counts.
bool i8_supported(int N);
int64_t i8_workspace_bytes(int64_t Q, int64_t H, int N);
cudaError_t launch_i8_encode_and_rank(const SearchScene *tab, int num_scenes, const int *qscene,
                                      const int *hscene, int64_t Qtot, int64_t Htot,
                                      int64_t tiles_total, int N, void *ws, int *nwide, int *hwide,
                                      int *wn_list, int *wh_list, int *counts,
                                      const int *nflags, const int64_t *dtrue, int *rank,
                                      unsigned long long *best, cudaStream_t st);

// Carve 256-byte aligned sub-buffers out of one workspace allocation.
struct Carver {
  char *base;
  int64_t off = 0;
  constexpr Carver() : base(nullptr) {}  // sizing only: take() returns null pointers
  explicit Carver(void *b) : base(static_cast<char *>(b)) {}
  template <class T>
  constexpr T *take(int64_t count) {
    off = (off + 255) & ~int64_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * int64_t(sizeof(T));
    return p;
  }
};

// Items per block of the generation's bucket scan.
constexpr int kGenScanItems = 2048;

// Hashed buckets used for a scene of nt triangles (a power of two in [2^10, 2^22]).
__host__ __device__ constexpr uint32_t generate_bucket_count(int64_t nt) {
  uint32_t b = 1024;
  while (b < (uint64_t)nt && b < (1u << 22)) b <<= 1;
  return b;
}

// Generation workspace of a batch (the layout that bin_triangles carves, plus alignment slack).
constexpr int64_t generate_batch_workspace_bytes(int num_scenes, int64_t total_tris,
                                                 int64_t total_buckets) {
  Carver c;
  c.take<GenScene>(num_scenes);
  c.take<int>(total_buckets);                      // counts
  c.take<int>(total_buckets + 1);                  // starts
  c.take<int>(total_buckets / kGenScanItems + 2);  // scan partials
  c.take<uint32_t>(total_tris);                    // bucket of each triangle
  c.take<int>(total_tris);                         // slot within its bucket
  c.take<float4>(4 * total_tris);                  // records
  c.take<int>(8 * (int64_t)num_scenes);            // per-scene box of triangle centres
  c.take<float4>((total_tris + 31) / 32);          // bounding spheres of 32-record chunks
  c.take<float4>((total_tris + 1023) / 1024);      // bounding spheres of 1024-record groups
  return c.off + 256;
}

// Workspace of a single-scene generation (also used by the clutter measure and spin images).
constexpr int64_t generate_workspace_bytes(int64_t num_triangles) {
  return generate_batch_workspace_bytes(1, num_triangles,
                                        (int64_t)generate_bucket_count(num_triangles) + 1);
}

__device__ __forceinline__ void set_status(int *status, int bits) { atomicOr(status, bits); }

// Number of kernels this library has enqueued in the process (for launch accounting).
void count_launches(int64_t n);

// Clears the calling thread's last-error text and checks the arguments of a generation call
// (as rici_generate does); returns RICI_OK or the error code, with its text recorded.
int begin_generate_call(const float *V, const float *Nrm, int64_t nv, const int32_t *T, int64_t nt,
                        const int32_t *O, int64_t no, float R, int32_t N, const uint16_t *out);
// Records `message` as the calling thread's last-error text and returns `code`.
int report_error(int code, const char *message);

// Device address of the status word on the current device.
cudaError_t status_word_address(int **address);

// The generation kernel's FP32 projection stage for n points (frame in FP64, rounded to FP32).
cudaError_t launch_project_fp32(const float *pts, int64_t n, const float *sv, const float *sn,
                                float *out, cudaStream_t st);

// Measured whole-device dp4a issue rate (instructions per second), for roofline peaks.
cudaError_t measure_dp4a_rate(cudaStream_t st, double *per_second);
// Measured whole-device mma.sync s8 rate (int8 multiply-adds per second), for roofline peaks.
cudaError_t measure_mma_s8_rate(cudaStream_t st, double *macs_per_second);

}  // namespace rici
