// Measured arithmetic-pipe peaks of this GPU (a measurement aid for the
// roofline figures; the paper has no counterpart): independent fused
// multiply-add chains in FP64 or FP32 on every SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/neno6.h"

namespace {

constexpr int kChains = 8;   // independent chains per thread
constexpr int kIters = 4096;  // FMAs per chain

// written only if a chain ends at an impossible value: keeps the chains live
__device__ double g_sink64;
__device__ float g_sink32;
__device__ __forceinline__ void sink(double v) { g_sink64 = v; }
__device__ __forceinline__ void sink(float v) { g_sink32 = v; }

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s < (T)0) sink(s);  // the chains stay positive: never taken
}

template <typename T>
int run(double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return NENO6_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return NENO6_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NENO6_ERR_CUDA;
  }
  // b slightly below 1 and c small keep every value finite and normal
  const T b = (T)0.999999, c = (T)1e-6;
  fma_chains_kernel<T><<<blocks, threads, 0, s>>>(b, c);  // warm-up
  cudaEventRecord(e0, s);
  fma_chains_kernel<T><<<blocks, threads, 0, s>>>(b, c);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.0f)) return NENO6_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)kIters * blocks * threads;
  *flops_per_s = flops / (ms * 1e-3);
  return NENO6_OK;
}

}  // namespace

extern "C" int neno6_pipe_peak(int which, double* flops_per_s, void* stream) {
  if (!flops_per_s || (which != 0 && which != 1)) return NENO6_ERR_ARG;
  return which == 0 ? run<double>(flops_per_s, (cudaStream_t)stream) : run<float>(flops_per_s, (cudaStream_t)stream);
}
