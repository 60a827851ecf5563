/*
 * rici.h — C ABI of the GB300 (sm_103a) RICI library.
 *
 * Radial Intersection Count Images (van Blokland & Theoharis, "Radial intersection count
 * image: a clutter resistant 3D shape descriptor", 2020): generation of uint16 count images
 * from a triangle mesh (Section 3.1) and search with the clutter-resistant distance
 * (Section 3.2, Listing 1, Eq. distanceFunctionExpression), ranking the true match as in the
 * clutterbox experiment (Section 4.1, tie rule of Section 4.2).
 *
 * Conventions for every call:
 *  - Array arguments are DEVICE pointers owned by the caller (for example torch CUDA tensor
 *    storage).  The library never frees or retains them after the call's work completes.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  All
 *    work is enqueued asynchronously on that stream; outputs are valid once it completes.
 *  - `workspace` is optional device scratch memory of at least the size returned by the
 *    matching *_workspace_size query, 256-byte aligned.  When it is NULL the library uses a
 *    per-device workspace of its own that grows on demand (cudaMalloc) and is released by
 *    rici_release_workspace().  A caller-provided workspace must not be used by another call
 *    that may run concurrently.
 *  - Return value: RICI_OK, or an error code for problems detectable on the host (invalid
 *    argument, CUDA launch error).  Errors found while the kernels run (an out-of-range
 *    triangle or match index, a non-finite coordinate) are OR-ed into a per-device status
 *    word that rici_sync_status() reads and clears.
 *  - Zero origins / triangles / needles are valid no-ops (images of a mesh without
 *    triangles are all zero).
 */
#ifndef RICI_H_
#define RICI_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RICI_API __attribute__((visibility("default")))
#else
#define RICI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Return and status codes (status bits may be OR-ed together). */
#define RICI_OK 0
#define RICI_ERR_INVALID_ARGUMENT 1   /* null pointer, negative count, bad resolution/radius */
#define RICI_ERR_INDEX_OUT_OF_RANGE 2 /* triangle, origin or true-match index out of range */
#define RICI_ERR_NONFINITE_INPUT 4    /* NaN or infinite vertex / normal coordinate */
#define RICI_ERR_OUT_TOO_LARGE 8      /* requested output exceeds the library's size cap */
#define RICI_ERR_CUDA 16              /* a CUDA runtime call failed */
#define RICI_ERR_WORKSPACE 32         /* caller workspace too small or misaligned */
#define RICI_ERR_TIMEOUT 64           /* a bounded device-side wait gave up */

/* Largest supported image resolution N (images are N x N). */
#define RICI_MAX_RESOLUTION 128

/* Generation modes (rici_generate_ex). */
#define RICI_GEN_DEFAULT 0   /* FP32 arithmetic; predicates inside the error band redone in FP64 */
#define RICI_GEN_FP64 1      /* every (triangle, layer) evaluated in FP64 (slow reference mode) */

/* Search modes (crss_search). */
#define RICI_SEARCH_DEFAULT 0   /* fastest exact form available: RICI_SEARCH_TENSOR where it
                                   applies (N in 8..128, powers of two), else CUDA cores */
#define RICI_SEARCH_CUDA_CORE 1 /* Listing 1 per pair on CUDA cores, early exit */
#define RICI_SEARCH_EXACT_SLOW 2 /* generic int64 per-pair kernel for every pair (test reference) */
#define RICI_SEARCH_TENSOR 3    /* exact fp16 tcgen05 GEMM of the expanded distance (N in 8..128,
                                   powers of two) for needles with every |delta| <= 127 and
                                   haystack images with every |delta| <= 45 and
                                   sum b^2 + 254 sum |b| < 2^24 (all partial sums exact in FP32);
                                   single-scene calls run the other int8-class pairs on the dense
                                   CUDA-core kernel, and pairs with |delta| > 127 (multi-scene
                                   calls: any pair outside the fp16 class) in exact int64 */
#define RICI_SEARCH_SPARSE 4    /* Listing 1 over each needle's non-zero delta words only (the
                                   positions where a != 0, Section 3.2), on CUDA cores: words
                                   heaviest first, early exit after every word; single-scene
                                   calls with N in {8,16,32,64,128} (other calls take the int64
                                   kernel); fastest when needles are sparse */
#define RICI_SEARCH_INT8_TC 5  /* exact int8 tensor-core GEMM of the expanded distance (warp-level
                                   mma.sync s8 -> s32, N in 8..128, powers of two): operands a, m
                                   and the haystack deltas b with b^2 split into two 7-bit limbs;
                                   pairs with |delta| > 127 on either side run in exact int64 on
                                   CUDA cores; single- and multi-scene calls */
#define RICI_SEARCH_AUTO 6      /* each needle ranked by the fp16 tensor-core form or by the
                                   sparse-needle form, chosen per needle on the device: the
                                   sparse form when at most a quarter of its 32-bit delta words
                                   hold a non-zero delta (N in 8..128, powers of two, single-scene
                                   calls; multi-scene calls take RICI_SEARCH_TENSOR) */
/* Test hook, OR-ed into RICI_SEARCH_TENSOR: one CTA of the tensor-core kernel withholds its
 * first tile load, so its bounded waits run out (about 2 s), RICI_ERR_TIMEOUT is raised in the
 * status word and the kernel returns; outputs of that call are unspecified. */
#define RICI_SEARCH_TEST_WITHHOLD_LOAD 0x100

/*
 * rici_generate — one RICI image per oriented point (Section 3.1).
 *
 *   vertices   [num_vertices][3] float32 positions.
 *   normals    [num_vertices][3] float32 normals; any positive length (the frame coefficients
 *              of Eq. rotationCoefficients normalise), zero selects the identity rotations.
 *   triangles  [num_triangles][3] int32 vertex indices.
 *   origins    [num_origins] int32 vertex indices: oriented point k is
 *              (vertices[origins[k]], normals[origins[k]]).
 *   support_radius  R > 0 and finite: circles have radii alpha_c = R(2c+1)/(2N) and sit in
 *              layers beta_r = R(2r+1-N)/(2N) along the normal, c, r in [0, N).
 *   resolution N in [1, RICI_MAX_RESOLUTION].
 *   out_images [num_origins][N][N] uint16, row r = layer beta_r, column c = radius alpha_c;
 *              bin (r, c) counts how many times circle (r, c) crosses the mesh surface,
 *              saturated at 65535.  Bit-identical to the FP64 brute-force definition.
 *
 * Errors: RICI_ERR_INVALID_ARGUMENT on the host; RICI_ERR_INDEX_OUT_OF_RANGE and
 * RICI_ERR_NONFINITE_INPUT in the status word (outputs are then unspecified).
 */
RICI_API int64_t rici_generate_workspace_size(int64_t num_vertices, int64_t num_triangles,
                                     int64_t num_origins, int32_t resolution);
RICI_API int rici_generate(const float *vertices, const float *normals, int64_t num_vertices,
                  const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                  int64_t num_origins, float support_radius, int32_t resolution,
                  uint16_t *out_images, void *workspace, int64_t workspace_bytes, void *stream);
/* As rici_generate with a mode (RICI_GEN_*) and optional device counters:
 * counters (NULL or device int64[4]) receives, added to its contents:
 *   [0] (origin, triangle) pairs fully processed after culling,
 *   [1] (origin, triangle, layer) items processed,
 *   [2] items re-evaluated in FP64 because a predicate fell inside the FP32 error band,
 *   [3] candidate (origin, triangle) pairs tested one by one by the spatial cull (those in
 *       32-triangle chunks whose bounding spheres passed). */
RICI_API int rici_generate_ex(const float *vertices, const float *normals, int64_t num_vertices,
                     const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                     int64_t num_origins, float support_radius, int32_t resolution,
                     uint16_t *out_images, int32_t mode, int64_t *counters, void *workspace,
                     int64_t workspace_bytes, void *stream);

/*
 * crss_search — clutter-resistant search (Listing 1, Eq. distanceFunctionExpression).
 *
 *   d(i, j) = sum over r in [0,N), c in [1,N) with a != 0 of (a - b)^2, where
 *   a = needle_i[r][c] - needle_i[r][c-1] and b = haystack_j[r][c] - haystack_j[r][c-1].
 *
 *   needles    [num_needles][N][N] uint16;  haystack [num_haystack][N][N] uint16.
 *   true_match [num_needles] int64 haystack index of needle i's true match, or NULL for i.
 *   out_rank   [num_needles] int32: #{j : d(i,j) < d(i, match_i)} (ties keep the best rank).
 *   out_true_distance [num_needles] int64 d(i, match_i), or NULL.
 *   out_top1   [num_needles] int32 smallest j with minimal d(i, j), or NULL.
 *   out_distances [num_needles][num_haystack] int64 full distance matrix, or NULL; rejected
 *              with RICI_ERR_OUT_TOO_LARGE when num_needles*num_haystack > 2^28.
 *   mode       RICI_SEARCH_*.
 * All outputs are exact (integer arithmetic).  num_haystack must be > 0 when
 * num_needles > 0.  An out-of-range true_match entry sets RICI_ERR_INDEX_OUT_OF_RANGE.
 */
RICI_API int64_t crss_search_workspace_size(int64_t num_needles, int64_t num_haystack,
                                   int32_t resolution, int32_t mode);
RICI_API int crss_search(const uint16_t *needles, int64_t num_needles, const uint16_t *haystack,
                int64_t num_haystack, int32_t resolution, const int64_t *true_match,
                int32_t *out_rank, int64_t *out_true_distance, int32_t *out_top1,
                int64_t *out_distances, int32_t mode, void *workspace, int64_t workspace_bytes,
                void *stream);

/* As crss_search with optional device counters (NULL or int64[4]), added to:
 *   [0] (pair, row) evaluations by the packed CUDA-core kernel (each row = N-1 positions;
 *       rows after a pair's early exit are not evaluated); with RICI_SEARCH_SPARSE,
 *       (pair, needle word) evaluations (each word = 4 positions of the needle, at least one
 *       of them non-zero),
 *   [1] pairs evaluated by the int64 kernel (pairs with a delta outside int8),
 *   [2] needle non-zero positions evaluated by the int64 kernel,
 *   [3] lane slots the packed kernel spent on those evaluations (32 per warp-wide iteration;
 *       [0] / [3] is its lane utilisation). */
RICI_API int crss_search_ex(const uint16_t *needles, int64_t num_needles,
                            const uint16_t *haystack, int64_t num_haystack, int32_t resolution,
                            const int64_t *true_match, int32_t *out_rank,
                            int64_t *out_true_distance, int32_t *out_top1,
                            int64_t *out_distances, int32_t mode, int64_t *counters,
                            void *workspace, int64_t workspace_bytes, void *stream);

/*
 * Multi-scene calls (batched run).  Every scene of a batch is processed by the same kernel
 * launches: one triangle binning pass, one generation grid over all scenes' oriented points,
 * one persistent tensor-core search over all scenes' tiles.  A batch call enqueues a fixed
 * sequence of kernels and copies, performs no host synchronisation and, with a caller
 * workspace, no allocation, so the sequence can be recorded into a CUDA graph and replayed.
 * The scene arrays are read on the host during the call only.
 */
typedef struct RiciGenerateScene {
  const float *vertices;   /* [num_vertices][3] */
  const float *normals;    /* [num_vertices][3] */
  int64_t num_vertices;
  const int32_t *triangles; /* [num_triangles][3] */
  int64_t num_triangles;
  const int32_t *origins;  /* [num_origins] vertex indices */
  int64_t num_origins;
  uint16_t *out_images;    /* [num_origins][N][N] */
} RiciGenerateScene;

/* Workspace for rici_generate_batch (-1 on invalid sizes). */
RICI_API int64_t rici_generate_batch_workspace_size(const RiciGenerateScene *scenes,
                                                    int32_t num_scenes, int32_t resolution);
/* rici_generate for every scene of the batch (same R and N; results identical to one
 * rici_generate call per scene). */
RICI_API int rici_generate_batch(const RiciGenerateScene *scenes, int32_t num_scenes,
                                 float support_radius, int32_t resolution, void *workspace,
                                 int64_t workspace_bytes, void *stream);

typedef struct RiciSearchScene {
  const uint16_t *needles;   /* [num_needles][N][N] */
  int64_t num_needles;
  const uint16_t *haystack;  /* [num_haystack][N][N] */
  int64_t num_haystack;
  const int64_t *true_match; /* [num_needles] scene-local haystack indices, or NULL for i */
  int32_t *out_rank;         /* [num_needles] */
  int64_t *out_true_distance; /* [num_needles] or NULL */
  int32_t *out_top1;         /* [num_needles] scene-local index, or NULL */
} RiciSearchScene;

/* Workspace for crss_search_batch (-1 on invalid sizes). */
RICI_API int64_t crss_search_batch_workspace_size(const RiciSearchScene *scenes,
                                                  int32_t num_scenes, int32_t resolution,
                                                  int32_t mode);
/* crss_search for every scene of the batch: each needle is ranked against its own scene's
 * haystack only.  RICI_SEARCH_TENSOR (or DEFAULT) runs one persistent tensor-core launch over all
 * scenes' tiles (pairs outside the fp16 class in exact int64), RICI_SEARCH_INT8_TC one int8
 * tensor-core launch over all scenes' tiles; RICI_SEARCH_CUDA_CORE and RICI_SEARCH_SPARSE run
 * the single-scene form scene after scene on the stream (one workspace sized for the largest
 * scene, no host synchronisation); RICI_SEARCH_EXACT_SLOW the int64 kernel over all scenes. */
RICI_API int crss_search_batch(const RiciSearchScene *scenes, int32_t num_scenes,
                               int32_t resolution, int32_t mode, void *workspace,
                               int64_t workspace_bytes, void *stream);

/*
 * rici_batch_run — the whole path for many scenes in one call: for every scene the needle
 * images (its target mesh alone), the haystack images (the whole scene) and the search of its
 * needles against its own haystack.  All needle and haystack images of all scenes come from one
 * rici_generate_batch launch sequence and the searches from one crss_search_batch sequence, in
 * stream order, so the call can be recorded into one CUDA graph and replayed.
 */
typedef struct RiciBatchScene {
  const float *vertices;   /* [num_vertices][3] the scene */
  const float *normals;    /* [num_vertices][3] */
  int64_t num_vertices;
  const int32_t *triangles; /* [num_triangles][3] */
  int64_t num_triangles;
  int64_t target_triangles; /* the target mesh is triangles [0, target_triangles) */
  const int32_t *needle_origins;   /* [num_needles] vertex indices (imaged with the target) */
  int64_t num_needles;
  const int32_t *haystack_origins; /* [num_haystack] vertex indices (imaged with the scene) */
  int64_t num_haystack;
  const int64_t *true_match; /* [num_needles] haystack index of needle i's match, or NULL: i */
  uint16_t *needle_images;   /* [num_needles][N][N] caller-owned */
  uint16_t *haystack_images; /* [num_haystack][N][N] caller-owned */
  int32_t *out_rank;          /* [num_needles] */
  int64_t *out_true_distance; /* [num_needles] or NULL */
  int32_t *out_top1;          /* [num_needles] or NULL */
} RiciBatchScene;

/* Workspace for rici_batch_run: the larger of its generation and search workspaces (the two
 * stages run one after the other on the stream and share it); -1 on invalid sizes. */
RICI_API int64_t rici_batch_run_workspace_size(const RiciBatchScene *scenes, int32_t num_scenes,
                                               int32_t resolution, int32_t mode);
/* Results identical to rici_generate for each scene's needles and haystack followed by
 * crss_search per scene; mode as for crss_search_batch. */
RICI_API int rici_batch_run(const RiciBatchScene *scenes, int32_t num_scenes,
                            float support_radius, int32_t resolution, int32_t mode,
                            void *workspace, int64_t workspace_bytes, void *stream);

/* rici_batch_run with the launch tuning of this call: `tuning` (see RiciTuning below) is in force
 * for this call only, on the calling thread (concurrent callers with different tunings do not
 * interfere, and the process-wide setting is neither read nor changed); NULL takes the
 * process-wide setting.  RICI_ERR_INVALID_ARGUMENT for a tuning out of range.  Results do not
 * depend on the tuning. */
typedef struct RiciTuning RiciTuning;
RICI_API int rici_batch_run_ex(const RiciBatchScene *scenes, int32_t num_scenes,
                               float support_radius, int32_t resolution, int32_t mode,
                               const RiciTuning *tuning, void *workspace, int64_t workspace_bytes,
                               void *stream);

/*
 * rici_clutter — the clutter measure of Eq. clutter (Section 4.1) per oriented point:
 * clutter = (A_all - A_object) / A_all, with A_all the surface area of the mesh inside the
 * oriented point's support volume and A_object the part of it on the object of interest.
 *
 *   vertices, normals, triangles, origins, support_radius  as for rici_generate.  The support
 *              volume is the cylinder of the image: radius R around the axis through the
 *              oriented point along its normal, heights |beta| <= R/2 along that axis.
 *   object_vertices  a triangle belongs to the object of interest when its first vertex index
 *              is below this count (the object's vertices come first, as in a clutterbox
 *              level); 0 counts no triangle, num_vertices every triangle.
 *   out_area_all, out_area_object  [num_origins] float64 device arrays (caller-owned): A_all
 *              and A_object, each the sum over triangles of the exact area of the triangle's
 *              part inside the volume (FP64 closed form: slab clip, then the projection's area
 *              within the disk over the cosine of the plane's tilt; planes within 1e-7 of
 *              parallel to the axis are cut by the two lines where they meet the cylinder).
 *   out_clutter  [num_origins] float64 device array, or NULL: Eq. clutter itself,
 *              (A_all - A_object) / A_all in FP64 (NaN where A_all = 0).
 * Workspace: rici_clutter_workspace_size bytes, or NULL to use the library's own.
 * Errors: as rici_generate (NaN outputs for an oriented point with a bad index or a
 * non-finite coordinate).
 */
RICI_API int64_t rici_clutter_workspace_size(int64_t num_triangles);
RICI_API int rici_clutter(const float *vertices, const float *normals, int64_t num_vertices,
                          const int32_t *triangles, int64_t num_triangles, const int32_t *origins,
                          int64_t num_origins, float support_radius, int64_t object_vertices,
                          double *out_area_all, double *out_area_object, double *out_clutter,
                          void *workspace, int64_t workspace_bytes, void *stream);

/*
 * rici_spin_images — spin images (Section 2.1, the descriptor the RICI is compared with) from
 * point samples of the mesh, with the projection of Section 3.1.1.
 *
 *   vertices, normals, triangles, origins, support_radius, resolution  as for rici_generate.
 *   samples_side  m in [1, 16]: m^2 samples per triangle, the centroids of the m^2 congruent
 *              triangles of a division of every side into m parts (uniform over its area).
 *   out_images [num_origins][N][N] float32 (caller-owned device memory): the plane is R wide
 *              and R high with the spin vertex at half height; bin (r, c) is centred at
 *              alpha_c = (c + 1/2) R/N, beta_r = (r + 1/2 - N/2) R/N; each sample with
 *              alpha^2 < R^2 and -R/2 <= beta < R/2 adds bilinear weights to the four bins
 *              around it (weight on a bin outside the image is dropped).  No support-angle
 *              filter.  The definition sums the weights as real numbers; this call forms
 *              positions, projection and weights in FP32 in a fixed order and sums each weight
 *              exactly as an integer number of units of 2^-24 (rounding error <= 2^-25 per
 *              weight; the sums do not depend on the order of the samples), so each bin differs
 *              from the FP64 definition by at most the rounding of those FP32 steps.
 * Workspace: rici_clutter_workspace_size bytes (the clutter measure's grid), or NULL.
 * Errors: as rici_generate (a zero image for an oriented point with a bad index or a
 * non-finite coordinate).
 */
RICI_API int rici_spin_images(const float *vertices, const float *normals, int64_t num_vertices,
                              const int32_t *triangles, int64_t num_triangles,
                              const int32_t *origins, int64_t num_origins, float support_radius,
                              int32_t resolution, int32_t samples_side, float *out_images,
                              void *workspace, int64_t workspace_bytes, void *stream);

/*
 * rici_generate_noalloc — rici_generate for callers that must not allocate device memory.
 * (An addition of this library; the paper has no counterpart.)
 *
 * Some callers cannot let a library call cudaMalloc or cudaFree: a service whose device
 * memory budget is fixed at start-up, a plugin host that owns the GPU allocator and offers
 * no scratch buffers, or a latency-critical loop where cudaFree's implicit device-wide
 * synchronisation would stall other streams.  This variant allocates nothing: its scratch
 * space is one 21 MiB array in device memory, compiled into the library, which every GPU that
 * loads the library holds until the process exits.  Arguments, outputs and results are those
 * of rici_generate (bit-identical images), without a workspace argument.
 *  - Accepts at most 262,144 triangles; larger meshes return RICI_ERR_OUT_TOO_LARGE.
 *  - The first call on a device looks up the array's device address with that device current;
 *    make that first call before any stream capture.
 *  - All calls share the one array: calls that overlap on the GPU (no ordering between their
 *    streams) race on it and produce wrong images.  Order them on one stream.
 *  - Device-side errors go to the same status word as rici_generate (rici_sync_status).
 */
RICI_API int rici_generate_noalloc(const float *vertices, const float *normals,
                                   int64_t num_vertices, const int32_t *triangles,
                                   int64_t num_triangles, const int32_t *origins,
                                   int64_t num_origins, float support_radius, int32_t resolution,
                                   uint16_t *out_images, void *stream);

/* Synchronise `stream`, then read and clear the per-device status word (RICI_ERR_* bits). */
RICI_API int rici_sync_status(void *stream, int32_t *device_status);

/* Release the library-owned workspace of the current device. */
RICI_API int rici_release_workspace(void);

/* Text for the last host-side error on the calling thread ("" if none). */
RICI_API const char *rici_last_error_string(void);

/* Number of CUDA kernels this library has enqueued in the calling process so far. */
RICI_API int64_t rici_kernel_launches(void);

/* ------------------------------------------------------------------ launch tuning
 * Launch shapes of the kernels.  None of them changes a result: images, distances, ranks and
 * top-1 are bit-identical for every valid setting; only the speed differs.  The setting is
 * process-wide (every device and stream) and is read when a call launches its kernels.  The
 * paper has no counterpart (it fixes one kernel configuration for its GPU). */
struct RiciTuning {
  int32_t gen_cells_per_reach; /* 2, 3 or 4: grid cells per triangle reach (the support
                                  sphere's radius plus the largest binned triangle's) of the
                                  clutter measure and spin images, which scan up to 7^3 cells
                                  around each oriented point (at most 3 per reach). Image
                                  generation sorts its triangles along a space-filling curve
                                  and culls them by bounding spheres of runs of 32 and 1024
                                  instead, and ignores this field. Default 2. */
  float gen_big_radius;        /* in [1/16, 1]: in the clutter measure and spin images,
                                  triangles whose bounding radius exceeds this fraction of the
                                  support sphere's radius are checked by every oriented point
                                  instead of being binned (image generation ignores it).
                                  Default 0.25. */
  int32_t gen_warps;           /* 4 or 8 warps per oriented point (image generation). Default 4. */
  int32_t tc_group_m;          /* 1..64: needle tiles of 128 that the tensor-core search sweeps
                                  together over the haystack (L2 reuse). Default 8. */
};

/* Sets the process-wide tuning; NULL restores the defaults.  RICI_ERR_INVALID_ARGUMENT when a
 * field is out of range (nothing changes then). */
RICI_API int rici_set_tuning(const RiciTuning *tuning);

/* Copies the tuning in force to *tuning (RICI_ERR_INVALID_ARGUMENT for NULL). */
RICI_API int rici_get_tuning(RiciTuning *tuning);

/* Autotuner of the batched run.  Runs rici_generate_batch on the given scenes under each candidate
 * generation setting (gen_warps in {4,8}; the other fields as in force, since image generation
 * reads no other field), one untimed warm-up and `repeats` (1..100)
 * runs timed with CUDA events on `stream`, and writes the fastest setting to *best and its mean
 * time in milliseconds to *best_ms (may be NULL).  The scenes' output images are written by every
 * run (with identical results).  Synchronises the stream; the tuning in force is restored, not
 * changed: apply *best with rici_set_tuning.  Arguments as for rici_generate_batch. */
RICI_API int rici_autotune_generate_batch(const RiciGenerateScene *scenes, int32_t num_scenes,
                                          float support_radius, int32_t resolution,
                                          void *workspace, int64_t workspace_bytes, void *stream,
                                          int32_t repeats, RiciTuning *best, float *best_ms);

/* The same for crss_search_batch in RICI_SEARCH_TENSOR form over tc_group_m in {2,4,8,16,32}. */
RICI_API int rici_autotune_search_batch(const RiciSearchScene *scenes, int32_t num_scenes,
                                        int32_t resolution, void *workspace,
                                        int64_t workspace_bytes, void *stream, int32_t repeats,
                                        RiciTuning *best, float *best_ms);

/* Projection of points into the frame of one oriented point with the generation kernel's FP32
 * stage, for checking that stage against an FP32 restatement: frame coefficients of Eq.
 * rotationCoefficients in FP64 (second pair on the rotated x, identity rule for zero pairs)
 * rounded to FP32, then Eqs. relativeLocation, firstRotation and secondRotation in FP32 with
 *   P' = P - S; P''x = fma(Nay, P'y, Nax*P'x); P''y = fma(Nax, P'y, -(Nay*P'x));
 *   Tx = fma(Nbz, P''x, -(Nbx*P'z)); Ty = P''y; Tz = fma(Nbx, P''x, Nbz*P'z)
 * (each product and sum rounded once).  points: device [n][3] float; spin_vertex, spin_normal:
 * device float[3]; out: device [n][3] float (Tx, Ty, Tz; alpha^2 = Tx^2 + Ty^2, beta = Tz).
 * Asynchronous on `stream`.  RICI_ERR_INVALID_ARGUMENT for a negative count or a null pointer
 * (n = 0 is a no-op), RICI_ERR_CUDA on a launch failure. */
RICI_API int rici_project_fp32(const float *points, int64_t num_points, const float *spin_vertex,
                               const float *spin_normal, float *out, void *stream);

/* Measures, on the current device and the given stream, how many dp4a instructions (four int8
 * multiply-adds into an int32 each; the arithmetic of the CUDA-core search) the whole GPU issues
 * per second, running independent accumulator chains on every SM; the result goes to
 * *dp4a_per_second.  Synchronises the stream; allocates and frees a small device buffer.
 * A measurement helper for roofline peaks: the paper has no counterpart.  Returns RICI_OK, or
 * RICI_ERR_INVALID_ARGUMENT for a null pointer, or RICI_ERR_CUDA. */
RICI_API int rici_measure_dp4a_rate(void *stream, double *dp4a_per_second);

/* Measures, on the current device and the given stream, how many int8 multiply-adds per second
 * the whole GPU performs through warp-level mma.sync m16n8k32 s8 x s8 -> s32 (the instruction of
 * RICI_SEARCH_INT8_TC), running independent accumulator chains on every SM; the result goes to
 * *int8_macs_per_second.  Synchronises the stream; allocates and frees a small device buffer.
 * A measurement helper for roofline peaks: the paper has no counterpart.  Returns RICI_OK,
 * RICI_ERR_INVALID_ARGUMENT for a null pointer, or RICI_ERR_CUDA. */
RICI_API int rici_measure_mma_s8_rate(void *stream, double *int8_macs_per_second);

/* Library version string. */
RICI_API const char *rici_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RICI_H_ */
