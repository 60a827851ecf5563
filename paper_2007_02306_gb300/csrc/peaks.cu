// Issue rate of dp4a, the instruction the CUDA-core search is built on, measured on the device.
//
// Each thread runs eight independent dp4a accumulator chains, so the measurement is bound by the
// pipe's throughput rather than by the latency of one chain.  The grid fills every SM several
// times over; each thread writes one word (the sum of its chains) so nothing is eliminated.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rici {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_dp4a_rate(int *out, int seed, int iters) {
  int acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = seed * (int)(threadIdx.x + i);
  const int x = seed ^ (int)threadIdx.x, y = seed + (int)blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = __dp4a(x + i, y, acc[i]);
    }
  }
  int s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t measure_dp4a_rate(cudaStream_t st, double *per_second) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int blocks = sms * 8, threads = 256, iters = 2000;
  int *out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(int) * (size_t)blocks * threads)) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.0f;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    k_dp4a_rate<<<blocks, threads, 0, st>>>(out, 3, iters);  // warm-up
    cudaEventRecord(e0, st);
    k_dp4a_rate<<<blocks, threads, 0, st>>>(out, 3, iters);
    cudaEventRecord(e1, st);
    count_launches(2);
    if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double n = (double)blocks * threads * iters * kUnroll * kChains;
  *per_second = ms > 0.0f ? n / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

}  // namespace rici
