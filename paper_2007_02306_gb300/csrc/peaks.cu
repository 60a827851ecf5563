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

// Integer tensor-core rate: every warp runs kMmaChains independent accumulator sets through
// mma.sync m16n8k32 s8 x s8 -> s32 (4,096 multiply-adds each) on register operands.
constexpr int kMmaChains = 8;

__global__ void __launch_bounds__(256) k_mma_s8_rate(int *out, int seed, int iters) {
  const uint32_t a0 = 0x01010101u * (uint32_t)(seed + threadIdx.x), a1 = a0 ^ 0x5a5a5a5au;
  const uint32_t a2 = a0 + 0x03030303u, a3 = a1 ^ 0x0f0f0f0fu;
  const uint32_t b0 = 0x02020202u ^ (uint32_t)blockIdx.x, b1 = b0 + 0x01010101u;
  int acc[kMmaChains][4];
#pragma unroll
  for (int c = 0; c < kMmaChains; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[c][e] = c + e;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
          "{%8, %9}, {%0, %1, %2, %3};"
          : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int c = 0; c < kMmaChains; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

// Times `launch` (one warm-up, one timed run) with events on st.
template <class F>
cudaError_t time_once(cudaStream_t st, F launch, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    launch();
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

cudaError_t measure_mma_s8_rate(cudaStream_t st, double *macs_per_second) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int blocks = sms * 4, threads = 256, iters = 4000;
  int *out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(int) * (size_t)blocks * threads)) != cudaSuccess) return e;
  float ms = 0.0f;
  e = time_once(st, [&] {
    k_mma_s8_rate<<<blocks, threads, 0, st>>>(out, 5, iters);
    count_launches(1);
  }, &ms);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double n = (double)blocks * (threads / 32) * iters * kMmaChains * 4096.0;
  *macs_per_second = ms > 0.0f ? n / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

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
