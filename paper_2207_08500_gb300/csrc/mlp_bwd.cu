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
// samples.  Per-CTA partial sums are reduced in a fixed order by a second
// kernel, so the result is deterministic.
#include <cmath>

#include "internal.h"

namespace neno6 {
namespace {

constexpr int kT = 128;        // samples per tile = threads per CTA
constexpr int kPitch = kT + 1;  // feature-major rows, padded against bank conflicts
// parameter offsets (per layer W[out][in] then b[out])
__host__ __device__ constexpr int wofs(int l) { return l == 0 ? 0 : l == 1 ? 448 : l == 2 ? 2528 : l == 3 ? 3056 : 3192; }
__host__ __device__ constexpr int wid(int l) { return l == 0 ? 6 : l == 1 ? 64 : l == 2 ? 32 : l == 3 ? 16 : l == 4 ? 8 : 4; }
// staged rows: inputs x0 (6) x1 (64) x2 (32) x3 (16) x4 (8); deltas d1..d5
constexpr int kX0 = 0, kX1 = 6, kX2 = 70, kX3 = 102, kX4 = 118;
constexpr int kD1 = 126, kD2 = 190, kD3 = 222, kD4 = 238, kD5 = 246, kRows = 250;
constexpr int kSmemFloats = kNetParams + kRows * kPitch;

__device__ __forceinline__ float softplus(float z) {  // log(1 + e^z), stable
  return fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z)));
}

__global__ void __launch_bounds__(kT) mlp_bwd_kernel(const double* __restrict__ X, const uint8_t* __restrict__ y,
                                                     long long n, const float* __restrict__ params,
                                                     float* __restrict__ partial, double* __restrict__ partial_loss) {
  extern __shared__ float sm[];
  float* W = sm;
  float* st = sm + kNetParams;
  const int t = threadIdx.x;
  for (int i = t; i < kNetParams; i += kT) W[i] = params[i];
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
    // ---- forward (Eq. (normalizainput), (reconstuction), (activationfunction))
    float x0[6], m = 1.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      x0[j] = live ? (float)X[s * 6 + j] : 0.0f;
      m = fmaxf(m, fabsf(x0[j]));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      x0[j] = x0[j] / m;
      st[(kX0 + j) * kPitch + t] = x0[j];
    }
    float h1[64];
#pragma unroll
    for (int o = 0; o < 64; ++o) {
      float a = W[wofs(0) + 384 + o];
#pragma unroll
      for (int i = 0; i < 6; ++i) a = fmaf(W[wofs(0) + o * 6 + i], x0[i], a);
      h1[o] = fmaxf(a, 0.0f);
      st[(kX1 + o) * kPitch + t] = h1[o];
    }
    float h2[32];
#pragma unroll
    for (int o = 0; o < 32; ++o) {
      float a = W[wofs(1) + 2048 + o];
#pragma unroll
      for (int i = 0; i < 64; ++i) a = fmaf(W[wofs(1) + o * 64 + i], h1[i], a);
      h2[o] = fmaxf(a, 0.0f);
      st[(kX2 + o) * kPitch + t] = h2[o];
    }
    float h3[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      float a = W[wofs(2) + 512 + o];
#pragma unroll
      for (int i = 0; i < 32; ++i) a = fmaf(W[wofs(2) + o * 32 + i], h2[i], a);
      h3[o] = fmaxf(a, 0.0f);
      st[(kX3 + o) * kPitch + t] = h3[o];
    }
    float h4[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      float a = W[wofs(3) + 128 + o];
#pragma unroll
      for (int i = 0; i < 16; ++i) a = fmaf(W[wofs(3) + o * 16 + i], h3[i], a);
      h4[o] = fmaxf(a, 0.0f);
      st[(kX4 + o) * kPitch + t] = h4[o];
    }
    // ---- output: loss and dL/dz = (sigma(z) - y) / (n S); ReLU masks of the
    // backward pass are re-read from the staged activations (fewer live
    // registers)
    asm volatile("" ::: "memory");
    float d5[4];
    const unsigned lab = live ? y[s] : 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float z = W[wofs(4) + 32 + k];
#pragma unroll
      for (int i = 0; i < 8; ++i) z = fmaf(W[wofs(4) + k * 8 + i], h4[i], z);
      const float yk = (float)((lab >> k) & 1u);
      const float sig = 1.0f / (1.0f + __expf(-z));
      // -[y log s + (1-y) log(1-s)] = softplus(z) - y z
      if (live) loss += (double)(softplus(z) - yk * z);
      d5[k] = live ? (sig - yk) * inv_nS : 0.0f;
      st[(kD5 + k) * kPitch + t] = d5[k];
    }
    // ---- backward: delta_l = (W_{l+1}^T delta_{l+1}) * relu'(pre-activation)
    float d4[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 4; ++k) a = fmaf(W[wofs(4) + k * 8 + i], d5[k], a);
      d4[i] = st[(kX4 + i) * kPitch + t] > 0.0f ? a : 0.0f;
      st[(kD4 + i) * kPitch + t] = d4[i];
    }
    float d3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) a = fmaf(W[wofs(3) + k * 16 + i], d4[k], a);
      d3[i] = st[(kX3 + i) * kPitch + t] > 0.0f ? a : 0.0f;
      st[(kD3 + i) * kPitch + t] = d3[i];
    }
    float d2[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 16; ++k) a = fmaf(W[wofs(2) + k * 32 + i], d3[k], a);
      d2[i] = st[(kX2 + i) * kPitch + t] > 0.0f ? a : 0.0f;
      st[(kD2 + i) * kPitch + t] = d2[i];
    }
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 32; ++k) a = fmaf(W[wofs(1) + k * 64 + i], d2[k], a);
      st[(kD1 + i) * kPitch + t] = st[(kX1 + i) * kPitch + t] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    // ---- parameter gradients over the tile: dW = delta^T x, db = sum delta
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int p = t + q * kT;
      if (p >= kNetParams) break;
      int l = 4;
      while (l > 0 && p < wofs(l)) --l;
      const int nin = wid(l), nout = wid(l + 1);
      const int r = p - wofs(l);
      const int drow = (l == 0 ? kD1 : l == 1 ? kD2 : l == 2 ? kD3 : l == 3 ? kD4 : kD5);
      const int xrow = (l == 0 ? kX0 : l == 1 ? kX1 : l == 2 ? kX2 : l == 3 ? kX3 : kX4);
      float a = 0.0f;
      if (r < nout * nin) {
        const float* dp = st + (drow + r / nin) * kPitch;
        const float* xp = st + (xrow + r % nin) * kPitch;
        for (int j = 0; j < kT; ++j) a = fmaf(dp[j], xp[j], a);
      } else {
        const float* dp = st + (drow + (r - nout * nin)) * kPitch;
        for (int j = 0; j < kT; ++j) a += dp[j];
      }
      acc[q] += a;
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

// grad[p] = sum_b partial[b][p] in block order; loss likewise (deterministic).
__global__ void mlp_bwd_reduce_kernel(const float* __restrict__ partial, const double* __restrict__ partial_loss,
                                      int blocks, long long n, float* __restrict__ grad, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNetParams) {
    float a = 0.0f;
    for (int b = 0; b < blocks; ++b) a += partial[(size_t)b * kNetParams + p];
    grad[p] = a;
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

size_t mlp_bwd_scratch_bytes(long long n) {
  const int b = mlp_bwd_blocks(n);
  return (size_t)b * kNetParams * sizeof(float) + (size_t)b * sizeof(double);
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
  mlp_bwd_reduce_kernel<<<(kNetParams + 255) / 256, 256, 0, s>>>(partial, partial_loss, blocks, n, grad, loss);
  return cudaGetLastError();
}

}  // namespace neno6
