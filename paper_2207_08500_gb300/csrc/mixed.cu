// Mixed-precision path of the NENO6 classifier and right-hand side on GB300:
// the classifier (Sec. 3.1, 6-64-32-16-8-4) runs on the 5th-generation tensor
// cores (tcgen05.mma, bf16 or fp16 operands, FP32 accumulators in tensor
// memory).
//
// Tensor-core MLP (one warpgroup per CTA): thread t owns row t of a 128-row
// batch, which is TMEM lane t and MMA row t.  Layer l's input (128 x K_l, K
// padded to a multiple of 16) sits in shared memory in the K-major canonical
// layout of tc.cuh; thread 0 issues the MMAs (D = A * W^T, N = layer width
// padded to 16) and commits them to an mbarrier; every thread waits (bounded),
// loads its row of the FP32 accumulator from TMEM, adds the FP32 bias, applies
// ReLU, rounds to bf16/fp16 and stores it as its row of the next layer's
// input.  TMEM columns: layer 1 [0,64), 2 [64,96), 3 [96,112), 4 [112,128),
// 5 [0,16) — 128 columns per CTA, so up to four CTAs share an SM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "internal.h"
#include "mlp_tc.cuh"
#include "tc.cuh"

namespace neno6 {
namespace {

using namespace tc;
using namespace tcmlp;

// Batched classifier (neno6_classify, mixed precision): persistent CTAs of
// 128 threads, one 128-row tile per iteration.  Normalisation (Eq.
// (normalizainput)) in FP32, then the tensor-core MLP; logit > 0 -> discard.
__global__ void __launch_bounds__(kMlpThreads) classify_mixed_kernel(const double* __restrict__ X,
                                                                      long long n, uint8_t* __restrict__ eta,
                                                                      double* __restrict__ logits,
                                                                      const uint8_t* __restrict__ net_image,
                                                                      int bf16, int* status) {
  __shared__ __align__(128) uint8_t s_net[kNetImageBytes];
  __shared__ __align__(128) uint8_t s_bufX[kBufXBytes];
  __shared__ __align__(128) uint8_t s_bufY[kBufYBytes];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int t = threadIdx.x;
  load_net_image(s_net, net_image);
  if (t == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    s_fail = 0;
  }
  if (t < 32) {
    tmem_alloc(&s_tmem, 64);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  MlpCtx c{s_net, s_bufX, s_bufY, &s_bar, s_tmem, 0u, bf16 != 0, &s_fail};
  const long long tiles = (n + 127) / 128;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long r = tile * 128 + t;
    float x[6];
    float m = 1.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      x[j] = r < n ? (float)X[r * 6 + j] : 0.0f;
      m = fmaxf(m, fabsf(x[j]));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) x[j] = x[j] / m;
    st_row8(s_bufY, t, 0, 16, pack2(x[0], x[1], c.bf16), pack2(x[2], x[3], c.bf16), pack2(x[4], x[5], c.bf16), 0u);
    st_row8(s_bufY, t, 8, 16, 0u, 0u, 0u, 0u);
    fence_async_smem();
    __syncthreads();
    float z[4];
    if (!mlp_tc(c, z)) {
      if (t == 0) atomicOr(status, 4);
      break;
    }
    if (r < n) {
      unsigned e = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) e |= (z[k] > 0.0f ? 1u : 0u) << k;
      eta[r] = (uint8_t)e;
      if (logits) {
#pragma unroll
        for (int k = 0; k < 4; ++k) logits[r * 4 + k] = (double)z[k];
      }
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (t < 32) tmem_dealloc(s_tmem, 64);
}

// Round a binary64 value to the nearest bf16 (ties to even) in one step.
uint16_t to_bf16_bits(double d) {
  if (d == 0.0) return std::signbit(d) ? 0x8000u : 0u;
  int e = std::ilogb(d);
  if (e < -133) e = -133;  // below the bf16 subnormal range: rounds to 0 / min
  const double scale = std::ldexp(1.0, e - 7);
  const double q = std::nearbyint(d / scale) * scale;  // 8 significant bits
  const float f = (float)q;                              // exact
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

uint16_t to_fp16_bits(double d) {
  __half h = __double2half(d);  // round to nearest even
  uint16_t u;
  std::memcpy(&u, &h, 2);
  return u;
}

}  // namespace

// Host: lay the FP64 master parameters out as the tensor-core image.
void build_net_image(const NetF64& net, bool bf16, uint8_t* img) {
  std::memset(img, 0, kNetImageBytes);
  auto put = [&](int off, int K, int n, int k, double w) {
    const uint16_t b = bf16 ? to_bf16_bits(w) : to_fp16_bits(w);
    std::memcpy(img + off + kmajor_offset(n, k, K), &b, 2);
  };
  const int widths[6] = {6, 64, 32, 16, 8, 4};
  const int boff[3] = {kNetImageB1, kNetImageB2, kNetImageB3};
  const int Kpad[3] = {16, 64, 32};
  const int bias_off[5] = {0, 64, 96, 112, 120};
  float* bias = reinterpret_cast<float*>(img + kNetImageBias);
  float* w4 = reinterpret_cast<float*>(img + kNetImageW4);
  float* w5 = reinterpret_cast<float*>(img + kNetImageW5);
  size_t p = 0;
  for (int l = 0; l < 5; ++l) {
    const int nin = widths[l], nout = widths[l + 1];
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) {
        const double w = net.p[p + (size_t)o * nin + i];
        if (l < 3) put(boff[l], Kpad[l], o, i, w);
        else if (l == 3) w4[o * 16 + i] = (float)w;
        else w5[o * 8 + i] = (float)w;
      }
    p += (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) bias[bias_off[l] + o] = (float)net.p[p + o];
    p += nout;
  }
}

cudaError_t launch_classify_mixed(const double* X, long long n, uint8_t* eta, double* logits,
                                  const uint8_t* net_image, bool bf16, int* status, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const long long tiles = (n + 127) / 128;
  const int blocks = (int)(tiles < 152 * 4 ? tiles : 152 * 4);
  // 16 KB of unused dynamic shared memory keeps residency at <= 4 CTAs per
  // SM, so the four 128-column TMEM allocations always fit.
  constexpr int kPadSmem = 16 * 1024;
  cudaError_t e = cudaFuncSetAttribute(classify_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPadSmem);
  if (e != cudaSuccess) return e;
  classify_mixed_kernel<<<blocks, kMlpThreads, kPadSmem, s>>>(X, n, eta, logits, net_image, bf16 ? 1 : 0,
                                                              status);
  return cudaGetLastError();
}

}  // namespace neno6
