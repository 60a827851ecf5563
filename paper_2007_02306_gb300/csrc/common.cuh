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
int64_t generate_workspace_bytes(int64_t num_triangles);
// Enqueue generation on `stream` using `ws` (>= generate_workspace_bytes, 256-aligned).
cudaError_t launch_generate(const GenerateArgs &a, void *ws, cudaStream_t stream);

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

// Tensor-core search (tc_search.cu): operand encoding + persistent tcgen05 GEMM with the rank /
// top-1 epilogue for narrow x narrow pairs.  Fills nwide/hwide and the wide lists/counts.
bool tc_supported(int N);
int64_t tc_workspace_bytes(int64_t Q, int64_t H, int N);
cudaError_t launch_tc_encode_and_rank(const uint16_t *needles, int64_t Q, const uint16_t *haystack,
                                      int64_t H, int N, void *ws, int *nwide, int *hwide,
                                      int *wn_list, int *wh_list, int *counts,
                                      const int *nflags, const int64_t *dtrue, int *rank,
                                      unsigned long long *best, int *status, cudaStream_t st);

// Carve 256-byte aligned sub-buffers out of one workspace allocation.
struct Carver {
  char *base;
  int64_t off = 0;
  explicit Carver(void *b) : base(static_cast<char *>(b)) {}
  template <class T>
  T *take(int64_t count) {
    off = (off + 255) & ~int64_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * int64_t(sizeof(T));
    return p;
  }
};

__device__ __forceinline__ void set_status(int *status, int bits) { atomicOr(status, bits); }

// Number of kernels this library has enqueued in the process (for launch accounting).
void count_launches(int64_t n);

// Device address of the status word on the current device.
cudaError_t status_word_address(int **address);

}  // namespace rici
