// Arithmetic throughput microbenchmark: the rates that bound the k-space
// kernels (FP32 fused multiply-adds, scalar and packed two-wide, FP64 fused
// multiply-adds, and the hardware base-2 exponential), measured on the
// device with CUDA events. Each thread runs kChains independent dependency
// chains so that the pipes, not the latencies, set the rate; the grid fills
// every SM several times over.
#include <cstdint>
#include <cuda_runtime.h>

#include "qslab.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) peak_ffma_kernel(int iters, float seed, float* sink) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = seed + (float)(threadIdx.x + j);
  const float a = 0.999999f, b = 1.0e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = fmaf(v[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  if (s == 1.2345678f) sink[blockIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) peak_ffma2_kernel(int iters, float seed, float* sink) {
  float2 v[kChains / 2];
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j)
    v[j] = make_float2(seed + (float)(threadIdx.x + 2 * j), seed + (float)(threadIdx.x + 2 * j + 1));
  const float2 a = make_float2(0.999999f, 0.999999f), b = make_float2(1.0e-7f, 1.0e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) v[j] = __ffma2_rn(v[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) s += v[j].x + v[j].y;
  if (s == 1.2345678f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) peak_dfma_kernel(int iters, double seed, double* sink) {
  double v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = seed + (double)(threadIdx.x + j);
  const double a = 0.999999, b = 1.0e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = fma(v[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  if (s == 1.2345678) sink[blockIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kThreads) peak_ex2_kernel(int iters, float seed, float* sink) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = -1.0e-3f * (seed + (float)j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = -ex2_approx(v[j]) * 1.0e-3f;
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  if (s == 1.2345678f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int qslab_measure_peaks(int device, double* out4, void* stream) {
  if (!out4) return QSLAB_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return QSLAB_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return QSLAB_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = sms * 8;
  float* sinkf = nullptr;
  double* sinkd = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = QSLAB_OK;
  if (cudaMalloc(&sinkf, sizeof(float) * blocks) != cudaSuccess ||
      cudaMalloc(&sinkd, sizeof(double) * blocks) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = QSLAB_ERR_ALLOC;
  }
  // (kernel, iterations, operations per thread-iteration)
  for (int which = 0; which < 4 && rc == QSLAB_OK; ++which) {
    const int iters = which == 2 ? 64 : 2048;      // FP64 is far slower on this part
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {            // rep 0 warms up
      cudaEventRecord(e0, st);
      switch (which) {
        case 0: peak_ffma_kernel<<<blocks, kThreads, 0, st>>>(iters, 1.0f, sinkf); break;
        case 1: peak_ffma2_kernel<<<blocks, kThreads, 0, st>>>(iters, 1.0f, sinkf); break;
        case 2: peak_dfma_kernel<<<blocks, kThreads, 0, st>>>(iters, 1.0, sinkd); break;
        default: peak_ex2_kernel<<<blocks, kThreads, 0, st>>>(iters, 1.0f, sinkf); break;
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = QSLAB_ERR_CUDA; break; }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      // lane operations: one FMA (or ex2) per chain and iteration; the packed
      // kernel does two per instruction
      const double ops = (double)blocks * kThreads * (double)iters * kChains;
      const double rate = ops / (ms * 1e-3);
      if (rep > 0 && rate > best) best = rate;
    }
    out4[which] = best;
  }
  if (cudaGetLastError() != cudaSuccess && rc == QSLAB_OK) rc = QSLAB_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sinkf);
  cudaFree(sinkd);
  return rc;
}
