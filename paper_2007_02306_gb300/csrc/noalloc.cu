// rici_generate_noalloc: RICI generation for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: a service whose device
// memory budget is fixed when it starts, a plugin host that owns the GPU allocator and hands
// out no scratch buffers, or a latency-critical loop where cudaFree's implicit device-wide
// synchronisation would stall work on other streams.  For them this entry point takes its
// scratch space from one statically sized device array compiled into the library instead
// of from a caller buffer or the library's on-demand workspace.
//
// The array lives in device memory of every GPU that loads the library until the process
// exits.  All calls share it: calls that overlap on the GPU (for example on two streams
// without ordering between them) race on it and give wrong images.  Each call resets the
// parts that must start from a fixed value (the bin counts, and the box of triangle centres,
// which starts empty) before its kernels use them; the rest is overwritten before it is read.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"

namespace rici {
namespace {

// Largest mesh accepted, and the scratch size it needs (generate_workspace_bytes of it).
constexpr int64_t kNoAllocMaxTriangles = 262144;
constexpr size_t kNoAllocScratchBytes = (size_t)21 << 20;  // 21 MiB

static_assert(generate_workspace_bytes(kNoAllocMaxTriangles) <= (int64_t)kNoAllocScratchBytes,
              "the scratch array must hold the workspace of the largest accepted mesh");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int *g_status_ptr[kMaxDevices];    // device address of the status word, per device

// Once per device, with that device current: resolve the device addresses of the scratch
// array and of the status word (host code may not use the array's name as a pointer).
cudaError_t noalloc_setup(int dev, void **scratch, int **status) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int *st = nullptr;
    e = status_word_address(&st);
    if (e != cudaSuccess) return e;
    g_status_ptr[dev] = st;
    g_scratch_ptr[dev] = p;
  }
  *scratch = g_scratch_ptr[dev];
  *status = g_status_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rici

using namespace rici;

extern "C" int rici_generate_noalloc(const float *vertices, const float *normals,
                                     int64_t num_vertices, const int32_t *triangles,
                                     int64_t num_triangles, const int32_t *origins,
                                     int64_t num_origins, float support_radius,
                                     int32_t resolution, uint16_t *out_images, void *stream) {
  int rc = begin_generate_call(vertices, normals, num_vertices, triangles, num_triangles, origins,
                               num_origins, support_radius, resolution, out_images);
  if (rc) return rc;
  // the scratch array has room for the workspace of at most kNoAllocMaxTriangles triangles
  if (num_triangles > kNoAllocMaxTriangles)
    return report_error(RICI_ERR_OUT_TOO_LARGE,
                        "rici_generate_noalloc accepts at most 262144 triangles");
  if (num_origins == 0) return RICI_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return report_error(RICI_ERR_CUDA, "rici_generate_noalloc: no usable current device");
  void *scratch = nullptr;
  int *status = nullptr;
  if (noalloc_setup(dev, &scratch, &status) != cudaSuccess)
    return report_error(RICI_ERR_CUDA, "rici_generate_noalloc: device address lookup failed");
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
  a.mode = RICI_GEN_DEFAULT;
  a.counters = nullptr;
  a.status = status;
  if (launch_generate(a, scratch, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return report_error(RICI_ERR_CUDA, "rici_generate_noalloc: launch failed");
  return RICI_OK;
}
