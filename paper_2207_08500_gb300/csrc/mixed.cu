// Mixed-precision path of the NENO6 classifier and right-hand side on GB300:
// the classifier (Sec. 3.1, 6-64-32-16-8-4) runs on the 5th-generation tensor
// cores (tcgen05.mma, bf16 or fp16 operands, FP32 accumulators in tensor
// memory).
//
// Tensor-core MLP (one warpgroup per CTA): thread t owns row t of a 128-row
// batch, which is TMEM lane t and MMA row t.  Layer 1's input (128 x 16, K
// padded) sits in shared memory in the K-major canonical layout of tc.cuh;
// layers 2-4 read their input from tensor memory, where the previous layer's
// epilogue writes it (two 16-bit values per 32-bit column) into columns that
// layer's accumulator has vacated.  Thread 0 issues the MMAs (D = A * W^T,
// N = layer width) and commits them to an mbarrier; every thread waits
// (bounded), loads its row of the FP32 accumulator from TMEM, applies ReLU,
// rounds to bf16/fp16 (one packed cvt per pair) and stores it as its row of
// the next layer's input.  The biases of layers 1 and 2 are accumulated by
// the tensor cores (constant-one input columns, see ones_col); the biases of
// layers 3-4 are added in FP32 in the epilogues, and layer 5 (8 -> 4) runs
// in FP32 on the CUDA cores.  64 TMEM columns per CTA.
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
// Dynamic shared memory requested at launch and never touched: it brings a
// CTA's shared memory to ~28 KB, so that eight are resident per SM (their
// 8 x 64 TMEM columns are exactly the SM's 512) and a ninth never is, whose
// allocation would wait.
constexpr int kResidencyPad = 14 * 1024;
// static shared memory of the kernel below: image, input tile, barrier, TMEM
// address, timeout flag
constexpr int kClassifySmem = kNetImageBytes + kBufYBytes + 16;

template <bool BF16, bool NARROW>
__global__ void __launch_bounds__(kMlpThreads) classify_mixed_kernel(const double* __restrict__ X,
                                                                      long long n, uint8_t* __restrict__ eta,
                                                                      double* __restrict__ logits,
                                                                      const uint8_t* __restrict__ net_image,
                                                                      int* status) {
  __shared__ __align__(128) uint8_t s_net[kNetImageBytes];
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
  MlpCtx c{s_net, s_bufY, &s_bar, s_tmem, 0u, BF16, &s_fail};
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
    store_input_row<BF16>(s_bufY, t, x);
    fence_async_smem();
    __syncthreads();
    float z[4];
    if (!(NARROW ? mlp_tc_narrow<BF16>(c, z) : mlp_tc<BF16>(c, z))) {
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

double from_16_bits(uint16_t b, bool bf16) {
  if (bf16) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
  }
  __half h;
  std::memcpy(&h, &b, 2);
  return (double)__half2float(h);
}

}  // namespace

// Host: lay the FP64 master parameters out as the tensor-core image.
void build_net_image(const NetF64& net, bool bf16, uint8_t* img) {
  std::memset(img, 0, kNetImageBytes);
  auto bits = [&](double w) { return bf16 ? to_bf16_bits(w) : to_fp16_bits(w); };
  auto put_bits = [&](int off, int K, int n, int k, uint16_t b) {
    std::memcpy(img + off + kmajor_offset(n, k, K), &b, 2);
  };
  // b = hi + mid + lo, each term the 16-bit rounding of what is left
  auto put_bias = [&](int off, int K, int n, double b) {
    for (int q = 0; q < 3; ++q) {
      const uint16_t h = bits(b);
      put_bits(off, K, n, ones_col(bf16) + q, h);
      b -= from_16_bits(h, bf16);
    }
  };
  // layer-1 weight w of output n, input i: hi in column i, lo = the 16-bit
  // rounding of w - hi in column 6 + i (bf16; fp16 keeps the single
  // rounding, lo = 0)
  auto put_w1 = [&](int off, int n, int i, double w) {
    const uint16_t h = bits(w);
    put_bits(off, 16, n, i, h);
    if (bf16) put_bits(off, 16, n, 6 + i, bits(w - from_16_bits(h, bf16)));
  };
  const int widths[6] = {6, 64, 32, 16, 8, 4};
  const int boff[4] = {kNetImageB1, kNetImageB2, kNetImageB3, kNetImageB4};
  const int Kpad[4] = {16, 64, 32, 16};
  float* bias = reinterpret_cast<float*>(img + kNetImageBias);
  float* w5t = reinterpret_cast<float*>(img + kNetImageW5);
  size_t p = 0;
  for (int l = 0; l < 5; ++l) {
    const int nin = widths[l], nout = widths[l + 1];
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) {
        const double w = net.p[p + (size_t)o * nin + i];
        if (l == 0) put_w1(boff[0], o, i, w);
        else if (l < 4) put_bits(boff[l], Kpad[l], o, i, bits(w));
        else w5t[i * 4 + o] = (float)w;
      }
    p += (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) {
      const double b = net.p[p + o];
      if (l == 0) put_bias(kNetImageB1, 16, o, b);
      else if (l == 1) put_bias(kNetImageB2b, 16, o, b);
      else bias[(l == 2 ? 0 : l == 3 ? 16 : 24) + o] = (float)b;
    }
    p += nout;
  }
}

// Host: the backward image (kBwd* layout).
void build_bwd_image(const NetF64& net, bool bf16, uint8_t* img) {
  std::memset(img, 0, kBwdImageBytes);
  auto put = [&](int off, int K, int n, int k, double w) {
    const uint16_t b = bf16 ? to_bf16_bits(w) : to_fp16_bits(w);
    std::memcpy(img + off + kmajor_offset(n, k, K), &b, 2);
  };
  // W3 [16 out][32 in] at 2528, W2 [32][64] at 448: B[n = in][k = out]
  for (int o = 0; o < 16; ++o)
    for (int i = 0; i < 32; ++i) put(kBwdBW3, 16, i, o, net.p[2528 + o * 32 + i]);
  for (int o = 0; o < 32; ++o)
    for (int i = 0; i < 64; ++i) put(kBwdBW2, 32, i, o, net.p[448 + o * 64 + i]);
  float* w4 = reinterpret_cast<float*>(img + kBwdW4);
  float* w5 = reinterpret_cast<float*>(img + kBwdW5);
  for (int q = 0; q < 8 * 16; ++q) w4[q] = (float)net.p[3056 + q];
  for (int q = 0; q < 4 * 8; ++q) w5[q] = (float)net.p[3192 + q];
}

// Host: the tensor-core image of the 6-32-32-32-4 network (kNarrow* layout).
void build_net_image_narrow(const NetF64& net, bool bf16, uint8_t* img) {
  std::memset(img, 0, kNetImageBytes);
  auto bits = [&](double w) { return bf16 ? to_bf16_bits(w) : to_fp16_bits(w); };
  auto put_bits = [&](int off, int K, int n, int k, uint16_t b) {
    std::memcpy(img + off + kmajor_offset(n, k, K), &b, 2);
  };
  auto put_bias = [&](int off, int n, double b) {
    for (int q = 0; q < 3; ++q) {
      const uint16_t h = bits(b);
      put_bits(off, 16, n, ones_col(bf16) + q, h);
      b -= from_16_bits(h, bf16);
    }
  };
  auto put_w1 = [&](int off, int n, int i, double w) {  // hi in column i, lo in 6 + i (bf16)
    const uint16_t h = bits(w);
    put_bits(off, 16, n, i, h);
    if (bf16) put_bits(off, 16, n, 6 + i, bits(w - from_16_bits(h, bf16)));
  };
  const int boff[3] = {kNarrowB1, kNarrowB2, kNarrowB3};
  const int Kpad[3] = {16, 32, 32};
  float* b3 = reinterpret_cast<float*>(img + kNarrowBias3);
  float* w4t = reinterpret_cast<float*>(img + kNarrowW4);
  size_t p = 0;
  for (int l = 0; l < 4; ++l) {
    const int nin = kNarrowWidths[l], nout = kNarrowWidths[l + 1];
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) {
        const double w = net.p[p + (size_t)o * nin + i];
        if (l == 0) put_w1(boff[0], o, i, w);
        else if (l < 3) put_bits(boff[l], Kpad[l], o, i, bits(w));
        else w4t[i * 4 + o] = (float)w;
      }
    p += (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) {
      const double b = net.p[p + o];
      if (l == 0) put_bias(kNarrowB1, o, b);
      else if (l == 1) put_bias(kNarrowB2b, o, b);
      else if (l == 2) b3[o] = (float)b;
      else w4t[128 + o] = (float)b;
    }
    p += nout;
  }
}

cudaError_t launch_classify_mixed(const double* X, long long n, uint8_t* eta, double* logits,
                                  const uint8_t* net_image, bool bf16, bool narrow, int* status,
                                  cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const long long tiles = (n + 127) / 128;
  // shared memory per CTA (128-byte units plus the 1 KB per-CTA reserve)
  // admits eight CTAs to the SM's 228 KB and never nine (kResidencyPad)
  constexpr int kPerCta = (kClassifySmem + kResidencyPad + 127) / 128 * 128 + 1024;
  static_assert(8 * kPerCta <= 228 * 1024, "eight resident CTAs");
  static_assert(9 * kPerCta > 228 * 1024, "nine resident CTAs would oversubscribe TMEM");
  static_assert(kClassifySmem + kResidencyPad <= 48 * 1024, "no opt-in needed");
  const int blocks = (int)(tiles < 152 * 8 ? tiles : 152 * 8);
  if (narrow) {
    if (bf16)
      classify_mixed_kernel<true, true><<<blocks, kMlpThreads, kResidencyPad, s>>>(X, n, eta, logits, net_image,
                                                                                  status);
    else
      classify_mixed_kernel<false, true><<<blocks, kMlpThreads, kResidencyPad, s>>>(X, n, eta, logits, net_image,
                                                                                   status);
  } else if (bf16) {
    classify_mixed_kernel<true, false><<<blocks, kMlpThreads, kResidencyPad, s>>>(X, n, eta, logits, net_image,
                                                                                 status);
  } else {
    classify_mixed_kernel<false, false><<<blocks, kMlpThreads, kResidencyPad, s>>>(X, n, eta, logits, net_image,
                                                                                  status);
  }
  return cudaGetLastError();
}

}  // namespace neno6
