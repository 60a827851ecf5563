// extern "C" entry points of librici: argument validation, workspace management and the
// per-device status word.  The compute stages live in generate.cu and search.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace rici {
namespace {

__device__ int g_status;  // OR of RICI_ERR_* bits raised by kernels on this device

thread_local std::string t_last_error;
std::atomic<int64_t> g_launches{0};

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *where) {
  return fail(RICI_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

struct DeviceState {
  void *ws = nullptr;
  int64_t ws_bytes = 0;
  int *status = nullptr;
};

std::mutex g_mu;
std::vector<DeviceState> g_dev;

// Per-device state (status word address, library workspace); call with the device current.
int device_state(DeviceState **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
  DeviceState &d = g_dev[dev];
  if (!d.status) {
    e = cudaGetSymbolAddress((void **)&d.status, g_status);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
  }
  *out = &d;
  return RICI_OK;
}

// Library-owned workspace of at least `bytes`, grown on demand.
int library_workspace(DeviceState *d, int64_t bytes, void **ws) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (d->ws_bytes < bytes) {
    if (d->ws) {
      cudaError_t e = cudaFree(d->ws);
      d->ws = nullptr;
      d->ws_bytes = 0;
      if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    cudaError_t e = cudaMalloc(&d->ws, (size_t)bytes);
    if (e != cudaSuccess) {
      d->ws = nullptr;
      return cuda_fail(e, "cudaMalloc(workspace)");
    }
    d->ws_bytes = bytes;
  }
  *ws = d->ws;
  return RICI_OK;
}

int resolve_workspace(DeviceState *d, void *user, int64_t user_bytes, int64_t need, void **ws) {
  if (user) {
    if (user_bytes < need)
      return fail(RICI_ERR_WORKSPACE, "workspace too small: %lld < %lld bytes",
                  (long long)user_bytes, (long long)need);
    if (reinterpret_cast<uintptr_t>(user) & 255)
      return fail(RICI_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    *ws = user;
    return RICI_OK;
  }
  return library_workspace(d, need, ws);
}

int check_generate_args(const float *V, const float *Nrm, int64_t nv, const int32_t *T, int64_t nt,
                        const int32_t *O, int64_t no, float R, int32_t N, const uint16_t *out) {
  if (nv < 0 || nt < 0 || no < 0) return fail(RICI_ERR_INVALID_ARGUMENT, "negative count");
  if (N < 1 || N > RICI_MAX_RESOLUTION)
    return fail(RICI_ERR_INVALID_ARGUMENT, "resolution must be in [1, %d]", RICI_MAX_RESOLUTION);
  if (!(R > 0.0f) || !isfinite(R))
    return fail(RICI_ERR_INVALID_ARGUMENT, "support_radius must be positive and finite");
  if (nt > 0 && (!T || !V)) return fail(RICI_ERR_INVALID_ARGUMENT, "null triangles/vertices");
  if (no > 0 && (!O || !V || !Nrm || !out))
    return fail(RICI_ERR_INVALID_ARGUMENT, "null origins/vertices/normals/output");
  if (no > 0 && nv == 0) return fail(RICI_ERR_INVALID_ARGUMENT, "origins given without vertices");
  if (nt > (int64_t(1) << 31) - 2 || nv > (int64_t(1) << 31) - 2)
    return fail(RICI_ERR_OUT_TOO_LARGE, "more than 2^31-2 triangles or vertices");
  return RICI_OK;
}

}  // namespace

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int begin_generate_call(const float *V, const float *Nrm, int64_t nv, const int32_t *T, int64_t nt,
                        const int32_t *O, int64_t no, float R, int32_t N, const uint16_t *out) {
  t_last_error.clear();
  return check_generate_args(V, Nrm, nv, T, nt, O, no, R, N, out);
}

int report_error(int code, const char *message) { return fail(code, "%s", message); }

cudaError_t status_word_address(int **address) {
  return cudaGetSymbolAddress((void **)address, g_status);
}

}  // namespace rici

namespace rici {
namespace {
std::mutex g_tune_mu;
const Tuning kDefaultTuning = {2, 0.25f, 4, 8};
Tuning g_tuning = kDefaultTuning;
// A tuning in force for the calling thread only (a per-call tuning or an autotuner's candidate);
// null: the process-wide setting.
thread_local const Tuning *t_tuning_override = nullptr;

// Puts `t` in force for the calling thread until the guard ends (the previous override returns).
struct TuningOverride {
  const Tuning *prev;
  explicit TuningOverride(const Tuning *t) : prev(t_tuning_override) { t_tuning_override = t; }
  ~TuningOverride() { t_tuning_override = prev; }
};

bool tuning_valid(const RiciTuning &t) {
  return (t.gen_cells_per_reach >= 2 && t.gen_cells_per_reach <= 4) &&
         t.gen_big_radius >= 0.0625f && t.gen_big_radius <= 1.0f &&
         (t.gen_warps == 4 || t.gen_warps == 8) && t.tc_group_m >= 1 && t.tc_group_m <= 64;
}

RiciTuning to_public(const Tuning &t) {
  RiciTuning r;
  memset(&r, 0, sizeof(r));
  r.gen_cells_per_reach = t.gen_cells_per_reach;
  r.gen_big_radius = t.gen_big_radius;
  r.gen_warps = t.gen_warps;
  r.tc_group_m = t.tc_group_m;
  return r;
}

Tuning from_public(const RiciTuning &r) {
  return Tuning{r.gen_cells_per_reach, r.gen_big_radius, r.gen_warps, r.tc_group_m};
}

void store_tuning(const Tuning &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuning = t;
}

// Times `run` under each candidate tuning (one untimed warm-up, then `repeats` timed runs with
// CUDA events on the stream) and reports the fastest.  The tuning in force before the call is
// restored whatever happens.
template <class Run>
int autotune(const std::vector<Tuning> &cands, int32_t repeats, void *stream, Run run,
             RiciTuning *best, float *best_ms) {
  if (!best) return fail(RICI_ERR_INVALID_ARGUMENT, "null output pointer");
  if (repeats < 1 || repeats > 100) return fail(RICI_ERR_INVALID_ARGUMENT, "repeats in [1, 100]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Tuning saved = current_tuning();
  TuningOverride guard(nullptr);  // candidates below are in force for this thread only
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  int rc = RICI_OK;
  float best_t = 0.0f;
  Tuning best_c = saved;
  for (size_t i = 0; i < cands.size() && rc == RICI_OK; ++i) {
    t_tuning_override = &cands[i];
    if ((rc = run()) != RICI_OK) break;
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
    for (int r = 0; r < repeats && rc == RICI_OK; ++r) rc = run();
    if (rc != RICI_OK) break;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "event sync"); break; }
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) { rc = cuda_fail(e, "elapsed"); break; }
    ms /= (float)repeats;
    if (i == 0 || ms < best_t) {
      best_t = ms;
      best_c = cands[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RICI_OK) return rc;
  *best = to_public(best_c);
  if (best_ms) *best_ms = best_t;
  return RICI_OK;
}
}  // namespace

Tuning current_tuning() {
  if (t_tuning_override) return *t_tuning_override;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tuning;
}
}  // namespace rici

using namespace rici;

extern "C" {

int64_t rici_generate_workspace_size(int64_t num_vertices, int64_t num_triangles,
                                     int64_t num_origins, int32_t resolution) {
  (void)num_vertices;
  (void)num_origins;
  (void)resolution;
  if (num_triangles < 0) return -1;
  return generate_workspace_bytes(num_triangles);
}

int rici_generate_ex(const float *vertices, const float *normals, int64_t num_vertices,
                     const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                     int64_t num_origins, float support_radius, int32_t resolution,
                     uint16_t *out_images, int32_t mode, int64_t *counters, void *workspace,
                     int64_t workspace_bytes, void *stream) {
  t_last_error.clear();
  int rc = check_generate_args(vertices, normals, num_vertices, triangles, num_triangles, origins,
                               num_origins, support_radius, resolution, out_images);
  if (rc) return rc;
  if (mode != RICI_GEN_DEFAULT && mode != RICI_GEN_FP64)
    return fail(RICI_ERR_INVALID_ARGUMENT, "unknown generation mode %d", mode);
  if (num_origins == 0) return RICI_OK;
  DeviceState *d = nullptr;
  if ((rc = device_state(&d))) return rc;
  void *ws = nullptr;
  if ((rc = resolve_workspace(d, workspace, workspace_bytes,
                              generate_workspace_bytes(num_triangles), &ws)))
    return rc;
  GenerateArgs a;
  a.vertices = vertices;
  a.normals = normals;
  a.num_vertices = num_vertices;
  a.triangles = triangles;
  a.num_triangles = num_triangles;
  a.origins = origins;
  a.num_origins = num_origins;
  a.support_radius = support_radius;
  a.resolution = resolution;
  a.out_images = out_images;
  a.mode = mode;
  a.counters = counters;
  a.status = d->status;
  cudaError_t e = launch_generate(a, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rici_generate launch");
  return RICI_OK;
}

int64_t rici_clutter_workspace_size(int64_t num_triangles) {
  if (num_triangles < 0) return -1;
  return generate_workspace_bytes(num_triangles);
}

int rici_clutter(const float *vertices, const float *normals, int64_t num_vertices,
                 const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                 int64_t num_origins, float support_radius, int64_t object_vertices,
                 double *out_area_all, double *out_area_object, double *out_clutter,
                 void *workspace,
                 int64_t workspace_bytes, void *stream) {
  t_last_error.clear();
  // the generation checks, with the resolution of a valid call and a stand-in output pointer
  int rc = check_generate_args(vertices, normals, num_vertices, triangles, num_triangles,
                               origins, num_origins, support_radius, 1,
                               reinterpret_cast<const uint16_t *>(out_area_all));
  if (rc) return rc;
  if (num_origins > 0 && !out_area_object)
    return fail(RICI_ERR_INVALID_ARGUMENT, "null out_area_object");
  if (object_vertices < 0) return fail(RICI_ERR_INVALID_ARGUMENT, "negative object_vertices");
  if (num_origins == 0) return RICI_OK;
  DeviceState *d = nullptr;
  if ((rc = device_state(&d))) return rc;
  void *ws = nullptr;
  if ((rc = resolve_workspace(d, workspace, workspace_bytes,
                              generate_workspace_bytes(num_triangles), &ws)))
    return rc;
  ClutterArgs a;
  a.vertices = vertices;
  a.normals = normals;
  a.num_vertices = num_vertices;
  a.triangles = triangles;
  a.num_triangles = num_triangles;
  a.origins = origins;
  a.num_origins = num_origins;
  a.support_radius = support_radius;
  a.object_vertices = object_vertices;
  a.out_area_all = out_area_all;
  a.out_area_object = out_area_object;
  a.out_clutter = out_clutter;
  a.status = d->status;
  cudaError_t e = launch_clutter(a, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rici_clutter launch");
  return RICI_OK;
}

int rici_spin_images(const float *vertices, const float *normals, int64_t num_vertices,
                     const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                     int64_t num_origins, float support_radius, int32_t resolution,
                     int32_t samples_side, float *out_images, void *workspace,
                     int64_t workspace_bytes, void *stream) {
  t_last_error.clear();
  int rc = check_generate_args(vertices, normals, num_vertices, triangles, num_triangles,
                               origins, num_origins, support_radius, resolution,
                               reinterpret_cast<const uint16_t *>(out_images));
  if (rc) return rc;
  if (samples_side < 1 || samples_side > 16)
    return fail(RICI_ERR_INVALID_ARGUMENT, "samples_side must be in [1, 16]");
  if (num_origins == 0) return RICI_OK;
  DeviceState *d = nullptr;
  if ((rc = device_state(&d))) return rc;
  void *ws = nullptr;
  if ((rc = resolve_workspace(d, workspace, workspace_bytes,
                              generate_workspace_bytes(num_triangles), &ws)))
    return rc;
  SpinArgs a;
  a.vertices = vertices;
  a.normals = normals;
  a.num_vertices = num_vertices;
  a.triangles = triangles;
  a.num_triangles = num_triangles;
  a.origins = origins;
  a.num_origins = num_origins;
  a.support_radius = support_radius;
  a.resolution = resolution;
  a.samples_side = samples_side;
  a.out_images = out_images;
  a.status = d->status;
  cudaError_t e = launch_spin(a, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rici_spin_images launch");
  return RICI_OK;
}

int rici_generate(const float *vertices, const float *normals, int64_t num_vertices,
                  const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                  int64_t num_origins, float support_radius, int32_t resolution,
                  uint16_t *out_images, void *workspace, int64_t workspace_bytes, void *stream) {
  return rici_generate_ex(vertices, normals, num_vertices, triangles, num_triangles, origins,
                          num_origins, support_radius, resolution, out_images, RICI_GEN_DEFAULT,
                          nullptr, workspace, workspace_bytes, stream);
}

int64_t crss_search_workspace_size(int64_t num_needles, int64_t num_haystack, int32_t resolution,
                                   int32_t mode) {
  if (num_needles < 0 || num_haystack < 0 || resolution < 1 ||
      resolution > RICI_MAX_RESOLUTION)
    return -1;
  return search_workspace_bytes(num_needles, num_haystack, resolution, mode);
}

int crss_search_ex(const uint16_t *needles, int64_t num_needles, const uint16_t *haystack,
                   int64_t num_haystack, int32_t resolution, const int64_t *true_match,
                   int32_t *out_rank, int64_t *out_true_distance, int32_t *out_top1,
                   int64_t *out_distances, int32_t mode, int64_t *counters, void *workspace,
                   int64_t workspace_bytes, void *stream) {
  t_last_error.clear();
  if (num_needles < 0 || num_haystack < 0) return fail(RICI_ERR_INVALID_ARGUMENT, "negative count");
  if (resolution < 2 || resolution > RICI_MAX_RESOLUTION)
    return fail(RICI_ERR_INVALID_ARGUMENT, "resolution must be in [2, %d]", RICI_MAX_RESOLUTION);
  const int base_mode = mode & 0xff;
  if ((base_mode != RICI_SEARCH_DEFAULT && base_mode != RICI_SEARCH_CUDA_CORE &&
       base_mode != RICI_SEARCH_EXACT_SLOW && base_mode != RICI_SEARCH_TENSOR &&
       base_mode != RICI_SEARCH_SPARSE && base_mode != RICI_SEARCH_INT8_TC &&
       base_mode != RICI_SEARCH_AUTO) ||
      (mode & ~(0xff | RICI_SEARCH_TEST_WITHHOLD_LOAD)) ||
      ((mode & RICI_SEARCH_TEST_WITHHOLD_LOAD) && base_mode != RICI_SEARCH_TENSOR))
    return fail(RICI_ERR_INVALID_ARGUMENT, "unknown search mode %d", mode);
  if (num_needles == 0) return RICI_OK;
  if (num_haystack == 0)
    return fail(RICI_ERR_INVALID_ARGUMENT, "needles given with an empty haystack");
  if (!needles || !haystack || !out_rank)
    return fail(RICI_ERR_INVALID_ARGUMENT, "null needles/haystack/out_rank");
  if (num_haystack > (int64_t(1) << 31) - 1 || num_needles > (int64_t(1) << 31) - 1)
    return fail(RICI_ERR_OUT_TOO_LARGE, "more than 2^31-1 needles or haystack images");
  if (out_distances && (double)num_needles * (double)num_haystack > (double)(int64_t(1) << 28))
    return fail(RICI_ERR_OUT_TOO_LARGE, "distance matrix larger than 2^28 entries");
  DeviceState *d = nullptr;
  int rc;
  if ((rc = device_state(&d))) return rc;
  void *ws = nullptr;
  if ((rc = resolve_workspace(d, workspace, workspace_bytes,
                              search_workspace_bytes(num_needles, num_haystack, resolution, mode),
                              &ws)))
    return rc;
  SearchArgs a;
  a.needles = needles;
  a.num_needles = num_needles;
  a.haystack = haystack;
  a.num_haystack = num_haystack;
  a.resolution = resolution;
  a.true_match = true_match;
  a.out_rank = out_rank;
  a.out_true_distance = out_true_distance;
  a.out_top1 = out_top1;
  a.out_distances = out_distances;
  a.mode = mode;
  a.counters = counters;
  a.status = d->status;
  cudaError_t e = launch_search(a, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "crss_search launch");
  return RICI_OK;
}

int crss_search(const uint16_t *needles, int64_t num_needles, const uint16_t *haystack,
                int64_t num_haystack, int32_t resolution, const int64_t *true_match,
                int32_t *out_rank, int64_t *out_true_distance, int32_t *out_top1,
                int64_t *out_distances, int32_t mode, void *workspace, int64_t workspace_bytes,
                void *stream) {
  return crss_search_ex(needles, num_needles, haystack, num_haystack, resolution, true_match,
                        out_rank, out_true_distance, out_top1, out_distances, mode, nullptr,
                        workspace, workspace_bytes, stream);
}

// ---------------------------------------------------------------- batched calls

static int build_gen_batch(const RiciGenerateScene *scenes, int32_t ns, int32_t N,
                           std::vector<GenScene> *out, GenerateBatch *b) {
  if (ns < 0 || (ns > 0 && !scenes)) return fail(RICI_ERR_INVALID_ARGUMENT, "bad scene array");
  if (N < 1 || N > RICI_MAX_RESOLUTION)
    return fail(RICI_ERR_INVALID_ARGUMENT, "resolution must be in [1, %d]", RICI_MAX_RESOLUTION);
  out->resize(ns);
  int64_t tri = 0, ori = 0, bkt = 0;
  for (int32_t i = 0; i < ns; ++i) {
    const RiciGenerateScene &g = scenes[i];
    int rc = check_generate_args(g.vertices, g.normals, g.num_vertices, g.triangles,
                                 g.num_triangles, g.origins, g.num_origins, 1.0f, N, g.out_images);
    if (rc) return fail(rc, "scene %d: %s", (int)i, t_last_error.c_str());
    GenScene &e = (*out)[i];
    e = GenScene{};
    e.V = g.vertices;
    e.Nrm = g.normals;
    e.tris = g.triangles;
    e.origins = g.origins;
    e.out = g.out_images;
    e.nv = g.num_vertices;
    e.nt = g.num_triangles;
    e.no = g.num_origins;
    e.tri_off = tri;
    e.origin_off = ori;
    e.bucket_off = bkt;
    e.nbuckets = generate_bucket_count(g.num_triangles);
    tri += g.num_triangles;
    ori += g.num_origins;
    bkt += (int64_t)e.nbuckets + 1;
  }
  if (tri > (int64_t(1) << 31) - 2 || bkt > (int64_t(1) << 31) - 2)
    return fail(RICI_ERR_OUT_TOO_LARGE, "batch too large: %lld triangles", (long long)tri);
  b->num_scenes = ns;
  b->total_tris = tri;
  b->total_origins = ori;
  b->total_buckets = bkt;
  b->N = N;
  return RICI_OK;
}

int64_t rici_generate_batch_workspace_size(const RiciGenerateScene *scenes, int32_t num_scenes,
                                           int32_t resolution) {
  std::vector<GenScene> tab;
  GenerateBatch b{};
  if (build_gen_batch(scenes, num_scenes, resolution, &tab, &b)) return -1;
  return generate_batch_workspace_bytes(num_scenes > 0 ? num_scenes : 1, b.total_tris,
                                        b.total_buckets);
}

int rici_generate_batch(const RiciGenerateScene *scenes, int32_t num_scenes, float support_radius,
                        int32_t resolution, void *workspace, int64_t workspace_bytes,
                        void *stream) {
  t_last_error.clear();
  if (!(support_radius > 0.0f) || !isfinite(support_radius))
    return fail(RICI_ERR_INVALID_ARGUMENT, "support_radius must be positive and finite");
  std::vector<GenScene> tab;
  GenerateBatch b{};
  int rc = build_gen_batch(scenes, num_scenes, resolution, &tab, &b);
  if (rc) return rc;
  if (b.total_origins == 0) return RICI_OK;
  DeviceState *d = nullptr;
  if ((rc = device_state(&d))) return rc;
  void *ws = nullptr;
  if ((rc = resolve_workspace(d, workspace, workspace_bytes,
                              generate_batch_workspace_bytes(num_scenes, b.total_tris,
                                                             b.total_buckets),
                              &ws)))
    return rc;
  b.R = support_radius;
  b.mode = RICI_GEN_DEFAULT;
  b.counters = nullptr;
  b.status = d->status;
  cudaError_t e = launch_generate_batch(tab.data(), b, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rici_generate_batch launch");
  return RICI_OK;
}

static int build_search_batch(const RiciSearchScene *scenes, int32_t ns, int32_t N, int32_t mode,
                              std::vector<SearchScene> *out, SearchBatch *b) {
  if (ns < 0 || (ns > 0 && !scenes)) return fail(RICI_ERR_INVALID_ARGUMENT, "bad scene array");
  if (N < 2 || N > RICI_MAX_RESOLUTION)
    return fail(RICI_ERR_INVALID_ARGUMENT, "resolution must be in [2, %d]", RICI_MAX_RESOLUTION);
  if (mode != RICI_SEARCH_DEFAULT && mode != RICI_SEARCH_CUDA_CORE &&
      mode != RICI_SEARCH_EXACT_SLOW && mode != RICI_SEARCH_TENSOR && mode != RICI_SEARCH_SPARSE &&
      mode != RICI_SEARCH_INT8_TC && mode != RICI_SEARCH_AUTO)
    return fail(RICI_ERR_INVALID_ARGUMENT, "unknown search mode %d", mode);
  out->resize(ns);
  int64_t q = 0, h = 0, hmax = 0, tiles = 0;
  for (int32_t i = 0; i < ns; ++i) {
    const RiciSearchScene &g = scenes[i];
    if (g.num_needles < 0 || g.num_haystack < 0)
      return fail(RICI_ERR_INVALID_ARGUMENT, "scene %d: negative count", (int)i);
    if (g.num_needles > 0 && (g.num_haystack == 0 || !g.needles || !g.haystack || !g.out_rank))
      return fail(RICI_ERR_INVALID_ARGUMENT, "scene %d: null buffer or empty haystack", (int)i);
    SearchScene &e = (*out)[i];
    e = SearchScene{};
    e.needles = g.needles;
    e.haystack = g.haystack;
    e.match = g.true_match;
    e.rank = g.out_rank;
    e.dtrue = g.out_true_distance;
    e.top1 = g.out_top1;
    e.Q = g.num_needles;
    e.H = g.num_needles > 0 ? g.num_haystack : 0;
    e.qoff = q;
    e.hoff = h;
    e.tile_off = tiles;
    search_tiles(e.Q, e.H, &e.tiles_m, &e.tiles_n);
    if (e.Q == 0) e.tiles_m = e.tiles_n = 0;
    q += e.Q;
    h += e.H;
    hmax = e.H > hmax ? e.H : hmax;
    tiles += (int64_t)e.tiles_m * e.tiles_n;
  }
  if (q > (int64_t(1) << 31) - 1 || h > (int64_t(1) << 31) - 1)
    return fail(RICI_ERR_OUT_TOO_LARGE, "more than 2^31-1 needles or haystack images in a batch");
  b->num_scenes = ns;
  b->Qtot = q;
  b->Htot = h;
  b->Hmax = hmax;
  b->tiles_total = tiles;
  b->N = N;
  b->mode = mode == RICI_SEARCH_DEFAULT ? RICI_SEARCH_TENSOR : mode;
  return RICI_OK;
}

// The CUDA-core dense and sparse-needle kernels work on one haystack, so a multi-scene batch in
// those forms runs scene by scene (each scene's launches on the same stream, reusing one
// workspace sized for the largest scene; no host synchronisation, so the sequence can still be
// recorded into a CUDA graph).  The tensor-core forms run every scene in one set of launches.
static bool per_scene_form(int mode, int num_scenes) {
  return num_scenes > 1 && (mode == RICI_SEARCH_CUDA_CORE || mode == RICI_SEARCH_SPARSE);
}

static int64_t batch_search_workspace(const std::vector<SearchScene> &tab, const SearchBatch &b,
                                      int32_t num_scenes, int32_t N) {
  if (per_scene_form(b.mode, num_scenes)) {
    int64_t m = 256;
    for (const SearchScene &s : tab) {
      if (s.Q == 0) continue;
      const int64_t w = search_workspace_bytes(s.Q, s.H, N, b.mode);
      m = w > m ? w : m;
    }
    return m;
  }
  return search_batch_workspace_bytes(num_scenes > 0 ? num_scenes : 1, b.Qtot, b.Htot, N, b.mode);
}

int64_t crss_search_batch_workspace_size(const RiciSearchScene *scenes, int32_t num_scenes,
                                         int32_t resolution, int32_t mode) {
  std::vector<SearchScene> tab;
  SearchBatch b{};
  if (build_search_batch(scenes, num_scenes, resolution, mode, &tab, &b)) return -1;
  return batch_search_workspace(tab, b, num_scenes, resolution);
}

int crss_search_batch(const RiciSearchScene *scenes, int32_t num_scenes, int32_t resolution,
                      int32_t mode, void *workspace, int64_t workspace_bytes, void *stream) {
  t_last_error.clear();
  std::vector<SearchScene> tab;
  SearchBatch b{};
  int rc = build_search_batch(scenes, num_scenes, resolution, mode, &tab, &b);
  if (rc) return rc;
  if (b.Qtot == 0) return RICI_OK;
  DeviceState *d = nullptr;
  if ((rc = device_state(&d))) return rc;
  void *ws = nullptr;
  if ((rc = resolve_workspace(d, workspace, workspace_bytes,
                              batch_search_workspace(tab, b, num_scenes, resolution), &ws)))
    return rc;
  b.counters = nullptr;
  b.status = d->status;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (per_scene_form(b.mode, num_scenes)) {
    for (const SearchScene &sc : tab) {
      if (sc.Q == 0) continue;
      SearchArgs a;
      a.needles = sc.needles;
      a.num_needles = sc.Q;
      a.haystack = sc.haystack;
      a.num_haystack = sc.H;
      a.resolution = resolution;
      a.true_match = sc.match;
      a.out_rank = sc.rank;
      a.out_true_distance = sc.dtrue;
      a.out_top1 = sc.top1;
      a.out_distances = nullptr;
      a.mode = b.mode;
      a.counters = nullptr;
      a.status = d->status;
      cudaError_t e = launch_search(a, ws, st);
      if (e != cudaSuccess) return cuda_fail(e, "crss_search_batch launch");
    }
    return RICI_OK;
  }
  cudaError_t e = launch_search_batch(tab.data(), b, ws, st, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "crss_search_batch launch");
  return RICI_OK;
}

namespace {
// The generation and search scene lists of a batched run: needle scenes (target alone) first,
// then haystack scenes.
int split_batch_run(const RiciBatchScene *scenes, int32_t num_scenes,
                    std::vector<RiciGenerateScene> *gen, std::vector<RiciSearchScene> *srch) {
  if (num_scenes < 0 || (num_scenes > 0 && !scenes))
    return fail(RICI_ERR_INVALID_ARGUMENT, "bad scene array");
  if (num_scenes > (1 << 29)) return fail(RICI_ERR_OUT_TOO_LARGE, "too many scenes");
  gen->resize(2 * (size_t)num_scenes);
  srch->resize((size_t)num_scenes);
  for (int32_t i = 0; i < num_scenes; ++i) {
    const RiciBatchScene &sc = scenes[i];
    if (sc.target_triangles < 0 || sc.target_triangles > sc.num_triangles)
      return fail(RICI_ERR_INVALID_ARGUMENT, "scene %d: target_triangles outside [0, %lld]", i,
                  (long long)sc.num_triangles);
    RiciGenerateScene &n = (*gen)[i];
    n.vertices = sc.vertices;
    n.normals = sc.normals;
    n.num_vertices = sc.num_vertices;
    n.triangles = sc.triangles;
    n.num_triangles = sc.target_triangles;
    n.origins = sc.needle_origins;
    n.num_origins = sc.num_needles;
    n.out_images = sc.needle_images;
    RiciGenerateScene &h = (*gen)[num_scenes + i];
    h = n;
    h.num_triangles = sc.num_triangles;
    h.origins = sc.haystack_origins;
    h.num_origins = sc.num_haystack;
    h.out_images = sc.haystack_images;
    RiciSearchScene &q = (*srch)[i];
    q.needles = sc.needle_images;
    q.num_needles = sc.num_needles;
    q.haystack = sc.haystack_images;
    q.num_haystack = sc.num_haystack;
    q.true_match = sc.true_match;
    q.out_rank = sc.out_rank;
    q.out_true_distance = sc.out_true_distance;
    q.out_top1 = sc.out_top1;
  }
  return RICI_OK;
}
}  // namespace

int64_t rici_batch_run_workspace_size(const RiciBatchScene *scenes, int32_t num_scenes,
                                      int32_t resolution, int32_t mode) {
  std::vector<RiciGenerateScene> gen;
  std::vector<RiciSearchScene> srch;
  if (split_batch_run(scenes, num_scenes, &gen, &srch)) return -1;
  const int64_t g = rici_generate_batch_workspace_size(gen.data(), 2 * num_scenes, resolution);
  const int64_t q = crss_search_batch_workspace_size(srch.data(), num_scenes, resolution, mode);
  if (g < 0 || q < 0) return -1;
  return g > q ? g : q;
}

int rici_batch_run(const RiciBatchScene *scenes, int32_t num_scenes, float support_radius,
                   int32_t resolution, int32_t mode, void *workspace, int64_t workspace_bytes,
                   void *stream) {
  t_last_error.clear();
  std::vector<RiciGenerateScene> gen;
  std::vector<RiciSearchScene> srch;
  int rc = split_batch_run(scenes, num_scenes, &gen, &srch);
  if (rc) return rc;
  if ((rc = rici_generate_batch(gen.data(), 2 * num_scenes, support_radius, resolution,
                                workspace, workspace_bytes, stream)))
    return rc;
  return crss_search_batch(srch.data(), num_scenes, resolution, mode, workspace, workspace_bytes,
                           stream);
}

int rici_batch_run_ex(const RiciBatchScene *scenes, int32_t num_scenes, float support_radius,
                      int32_t resolution, int32_t mode, const RiciTuning *tuning,
                      void *workspace, int64_t workspace_bytes, void *stream) {
  t_last_error.clear();
  if (!tuning)
    return rici_batch_run(scenes, num_scenes, support_radius, resolution, mode, workspace,
                          workspace_bytes, stream);
  if (!tuning_valid(*tuning))
    return fail(RICI_ERR_INVALID_ARGUMENT,
                "tuning out of range (cells per reach 2..4, big radius [1/16,1], warps 4|8, "
                "group 1..64)");
  const Tuning t = from_public(*tuning);
  TuningOverride guard(&t);
  return rici_batch_run(scenes, num_scenes, support_radius, resolution, mode, workspace,
                        workspace_bytes, stream);
}

int rici_sync_status(void *stream, int32_t *device_status) {
  DeviceState *d = nullptr;
  int rc;
  if ((rc = device_state(&d))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int v = 0;
  e = cudaMemcpy(&v, d->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  e = cudaMemset(d->status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "clear status");
  if (device_status) *device_status = v;
  return RICI_OK;
}

int rici_release_workspace(void) {
  DeviceState *d = nullptr;
  int rc;
  if ((rc = device_state(&d))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (d->ws) {
    cudaError_t e = cudaFree(d->ws);
    d->ws = nullptr;
    d->ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
  }
  return RICI_OK;
}

const char *rici_last_error_string(void) { return t_last_error.c_str(); }

int64_t rici_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int rici_project_fp32(const float *points, int64_t num_points, const float *spin_vertex,
                      const float *spin_normal, float *out, void *stream) {
  t_last_error.clear();
  if (num_points < 0) return fail(RICI_ERR_INVALID_ARGUMENT, "negative point count");
  if (num_points == 0) return RICI_OK;
  if (!points || !spin_vertex || !spin_normal || !out)
    return fail(RICI_ERR_INVALID_ARGUMENT, "null pointer");
  cudaError_t e = launch_project_fp32(points, num_points, spin_vertex, spin_normal, out,
                                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rici_project_fp32 launch");
  return RICI_OK;
}

int rici_measure_dp4a_rate(void *stream, double *dp4a_per_second) {
  if (!dp4a_per_second) return fail(RICI_ERR_INVALID_ARGUMENT, "null output pointer");
  cudaError_t e = measure_dp4a_rate(static_cast<cudaStream_t>(stream), dp4a_per_second);
  if (e != cudaSuccess) return cuda_fail(e, "dp4a rate");
  return RICI_OK;
}

int rici_measure_mma_s8_rate(void *stream, double *int8_macs_per_second) {
  t_last_error.clear();
  if (!int8_macs_per_second) return fail(RICI_ERR_INVALID_ARGUMENT, "null output pointer");
  cudaError_t e = measure_mma_s8_rate(static_cast<cudaStream_t>(stream), int8_macs_per_second);
  if (e != cudaSuccess) return cuda_fail(e, "mma.sync s8 rate");
  return RICI_OK;
}

const char *rici_version(void) { return "rici-gb300 0.1 (sm_103a)"; }

int rici_set_tuning(const RiciTuning *tuning) {
  if (!tuning) {
    store_tuning(kDefaultTuning);
    return RICI_OK;
  }
  if (!tuning_valid(*tuning))
    return fail(RICI_ERR_INVALID_ARGUMENT,
                "tuning out of range (cells per reach 2..4, big radius [1/16,1], warps 4|8, "
                "group 1..64)");
  store_tuning(from_public(*tuning));
  return RICI_OK;
}

int rici_get_tuning(RiciTuning *tuning) {
  if (!tuning) return fail(RICI_ERR_INVALID_ARGUMENT, "null output pointer");
  *tuning = to_public(current_tuning());
  return RICI_OK;
}

int rici_autotune_generate_batch(const RiciGenerateScene *scenes, int32_t num_scenes,
                                 float support_radius, int32_t resolution, void *workspace,
                                 int64_t workspace_bytes, void *stream, int32_t repeats,
                                 RiciTuning *best, float *best_ms) {
  t_last_error.clear();
  std::vector<Tuning> cands;
  const Tuning base = current_tuning();
  // image generation reads gen_warps only (its culling has no grid)
  for (int w : {4, 8})
    cands.push_back(Tuning{base.gen_cells_per_reach, base.gen_big_radius, w, base.tc_group_m});
  return autotune(
      cands, repeats, stream,
      [&]() {
        return rici_generate_batch(scenes, num_scenes, support_radius, resolution, workspace,
                                   workspace_bytes, stream);
      },
      best, best_ms);
}

int rici_autotune_search_batch(const RiciSearchScene *scenes, int32_t num_scenes,
                               int32_t resolution, void *workspace, int64_t workspace_bytes,
                               void *stream, int32_t repeats, RiciTuning *best, float *best_ms) {
  t_last_error.clear();
  std::vector<Tuning> cands;
  const Tuning base = current_tuning();
  for (int g : {2, 4, 8, 16, 32})
    cands.push_back(Tuning{base.gen_cells_per_reach, base.gen_big_radius, base.gen_warps, g});
  return autotune(
      cands, repeats, stream,
      [&]() {
        return crss_search_batch(scenes, num_scenes, resolution, RICI_SEARCH_TENSOR, workspace,
                                 workspace_bytes, stream);
      },
      best, best_ms);
}

}  // extern "C"
