// Gradient of the classifier's training loss (retraining the NENO6 network):
// the mean binary cross entropy of Eq. (Crossentropy),
//   L = -1/(n S) sum_s sum_k [ y log sigma(z) + (1-y) log(1 - sigma(z)) ],
// S = 4 outputs, with respect to every parameter (w^l, b^l) of the
// 6-64-32-16-8-4 ReLU network of Sec. 3.1, in FP32.
//
// Persistent CTAs of 128 threads take 128-sample tiles.  Per tile, one thread
// per sample runs the forward pass (weights broadcast from shared memory), the
// output delta dL/dz = (sigma(z) - y)/(n S) and the backward deltas, staging
// every layer's input and delta feature-major in shared memory; then each
// thread accumulates ~25 of the 3228 parameter gradients over the tile's
// samples, four per pass (independent chains, each in sample order).  Per-CTA partial sums are reduced in a fixed order by a second
// kernel, so the result is deterministic.
#include "internal.h"
#include "mlp_fb.cuh"

namespace neno6 {
namespace {

using namespace mlpfb;

constexpr int kT = 128;        // samples per tile = threads per CTA
constexpr int kPitch = kT + 1;  // feature-major rows, padded against bank conflicts
constexpr int kSmemFloats = kNetParams + (kRows + 1) * kPitch;  // W, staged rows, a row of ones

__global__ void __launch_bounds__(kT) mlp_bwd_kernel(const double* __restrict__ X, const uint8_t* __restrict__ y,
                                                     long long n, const float* __restrict__ params,
                                                     float* __restrict__ partial, double* __restrict__ partial_loss) {
  extern __shared__ float sm[];
  float* W = sm;
  float* st = sm + kNetParams;
  float* ones = st + kRows * kPitch;
  const int t = threadIdx.x;
  for (int i = t; i < kNetParams; i += kT) W[i] = params[i];
  for (int i = t; i < kPitch; i += kT) ones[i] = 1.0f;
  constexpr int kPer = (kNetParams + kT - 1) / kT;  // parameters owned by this thread
  float acc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) acc[q] = 0.0f;
  double loss = 0.0;
  const float inv_nS = (float)(1.0 / (4.0 * (double)n));
  __syncthreads();
  const long long tiles = (n + kT - 1) / kT;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long s = tile * kT + t;
    const bool live = s < n;
    float xr[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) xr[j] = live ? (float)X[s * 6 + j] : 0.0f;
    sample_fwd_bwd<kPitch>(W, st, t, live, xr, live ? y[s] : 0u, inv_nS, loss);
    __syncthreads();
    // ---- parameter gradients over the tile: dW = delta^T x, db = sum delta,
    // four parameters per pass over the samples
#pragma unroll
    for (int q = 0; q < kPer; q += 4) {
      float g4[4];
      param_grads<kPitch, 4>(st, ones, t + q * kT, kT, kT, g4);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (q + u < kPer) acc[q + u] += g4[u];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int p = t + q * kT;
    if (p < kNetParams) partial[(size_t)blockIdx.x * kNetParams + p] = acc[q];
  }
  // block loss (fixed-order tree in shared memory)
  __shared__ double sl[kT];
  sl[t] = loss;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if (t < w) sl[t] += sl[t + w];
    __syncthreads();
  }
  if (t == 0) partial_loss[blockIdx.x] = sl[0];
}

// grad[p] = scale * sum_b partial[b][p] in block order; loss likewise
// (deterministic).  scale is 1 for partial sums of deltas that carry the
// 1/(n S) of the mean, 1/(n S) for sums of unscaled deltas.
__global__ void mlp_bwd_reduce_kernel(const float* __restrict__ partial, const double* __restrict__ partial_loss,
                                      int blocks, long long n, float scale, float* __restrict__ grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNetParams) {
    float a = 0.0f;
    for (int b = 0; b < blocks; ++b) a += partial[(size_t)b * kNetParams + p];
    grad[p] = a * scale;
  }
  if (p == 0 && loss) {
    double l = 0.0;
    for (int b = 0; b < blocks; ++b) l += partial_loss[b];
    *loss = (float)(l / (4.0 * (double)n));
  }
}

}  // namespace

int mlp_bwd_blocks(long long n) {
  const long long tiles = (n + kT - 1) / kT;
  return (int)(tiles < 152 ? tiles : 152);
}

// Partial sums of up to 2 x 152 CTAs (the tensor-core kernel runs two per SM).
size_t mlp_bwd_scratch_bytes(long long n) {
  const long long tiles = (n + kT - 1) / kT;
  const size_t b = (size_t)(tiles < 2 * 152 ? tiles : 2 * 152);
  return b * kNetParams * sizeof(float) + b * sizeof(double);
}

cudaError_t launch_mlp_bwd(const double* X, const uint8_t* y, long long n, const float* params, float* grad,
                           float* loss, void* scratch, cudaStream_t s) {
  const int blocks = mlp_bwd_blocks(n);
  float* partial = static_cast<float*>(scratch);
  double* partial_loss = reinterpret_cast<double*>(static_cast<char*>(scratch) +
                                                   (size_t)blocks * kNetParams * sizeof(float));
  const size_t smem = (size_t)kSmemFloats * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_bwd_kernel<<<blocks, kT, smem, s>>>(X, y, n, params, partial, partial_loss);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_mlp_bwd_reduce(partial, partial_loss, blocks, n, 1.0f, grad, loss, s);
}

cudaError_t launch_mlp_bwd_reduce(const float* partial, const double* partial_loss, int blocks, long long n,
                                  float scale, float* grad, float* loss, cudaStream_t s) {
  mlp_bwd_reduce_kernel<<<(kNetParams + 255) / 256, 256, 0, s>>>(partial, partial_loss, blocks, n, scale, grad,
                                                                 loss);
  return cudaGetLastError();
}

}  // namespace neno6
