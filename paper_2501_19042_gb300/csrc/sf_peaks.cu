// Microbenchmarks of the float32-lane pipes that bound the fused forward:
// fused multiply-add throughput (FMA pipe) and reciprocal square root
// throughput (MUFU), each timed with CUDA events over a whole-GPU launch.
#include <cmath>

#include "sf_internal.cuh"

namespace {

constexpr int kChains = 8;       // independent dependency chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;  // 2048 threads per SM

__global__ void __launch_bounds__(kThreads) ffma_kernel(float* sink, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 1234.5f) sink[blockIdx.x] = s;   // never true for these inputs; keeps the work
}

__global__ void __launch_bounds__(kThreads) mufu_kernel(float* sink, int iters) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1.0f + (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = rsqrtf(x[j]);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 1234.5f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" sf_status sf_lane_peaks(int device, double* fma_per_s, double* mufu_per_s, double* lane_mhz) {
  if (!fma_per_s || !mufu_per_s || !lane_mhz) return SF_ERR_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return SF_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SF_ERR_CUDA;
  const int blocks = prop.multiProcessorCount * kBlocksPerSM;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(float) * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int fma_iters = 4096, mufu_iters = 512, reps = 5;
  double best_fma = 0.0, best_mufu = 0.0;
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    for (int rep = 0; rep <= reps && e == cudaSuccess; ++rep) {   // rep 0 warms up
      e = cudaEventRecord(e0);
      if (which == 0)
        ffma_kernel<<<blocks, kThreads>>>(sink, fma_iters, 0.999999f, 1e-7f);
      else
        mufu_kernel<<<blocks, kThreads>>>(sink, mufu_iters);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(e1);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess || rep == 0 || ms <= 0.0f) continue;
      const int iters = which == 0 ? fma_iters : mufu_iters;
      const double ops = (double)blocks * kThreads * iters * 4.0 * kChains;
      const double rate = ops / (ms * 1e-3);
      if (which == 0 && rate > best_fma) best_fma = rate;
      if (which == 1 && rate > best_mufu) best_mufu = rate;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return SF_ERR_CUDA;
  *fma_per_s = best_fma;
  *mufu_per_s = best_mufu;
  // the clock at which 128 FP32 lanes per SM, one FMA each per cycle, give
  // the measured rate
  *lane_mhz = best_fma / (128.0 * prop.multiProcessorCount) / 1e6;
  return SF_OK;
}
