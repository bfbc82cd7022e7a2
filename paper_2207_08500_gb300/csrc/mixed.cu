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
#include "tc.cuh"

namespace neno6 {
namespace {

using namespace tc;

constexpr int kMlpThreads = 128;
constexpr int kBufXBytes = 128 * 64 * 2;  // A2 (K = 64) / A4
constexpr int kBufYBytes = 128 * 32 * 2;  // A1 / A3 (K = 32) / A5

__device__ __forceinline__ uint32_t pack2(float a, float b, bool bf16) {
  if (bf16) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Store 8 consecutive K values (one core-matrix row) of row `row`.
__device__ __forceinline__ void st_row8(uint8_t* base, int row, int k0, int K, uint32_t a, uint32_t b,
                                        uint32_t c, uint32_t d) {
  const uint32_t addr = smem_u32(base + kmajor_offset(row, k0, K));
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

struct MlpCtx {
  const uint8_t* net;  // shared-memory image (kNetImage* layout)
  uint8_t* bufX;
  uint8_t* bufY;
  uint64_t* bar;
  uint32_t tmem;
  uint32_t phase;
  bool bf16;
};

// Issue one layer (thread 0): ksteps MMAs of K = 16 into TMEM column `col`.
__device__ __forceinline__ void issue_layer(const MlpCtx& c, const uint8_t* A, int K, int B_off, int N,
                                            int col) {
  const uint32_t sbo = (uint32_t)(K / 8) * 128u;
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(c.net + B_off);
  const uint32_t idesc = idesc_f16(128, N, c.bf16);
  tc_fence_after();
  for (int ks = 0; ks < K / 16; ++ks)
    mma_f16(c.tmem + (uint32_t)col, smem_desc(a0 + 256u * ks, 128u, sbo),
            smem_desc(b0 + 256u * ks, 128u, sbo), idesc, ks > 0 ? 1u : 0u);
  mma_commit(c.bar);
}

// Wait for the layer's MMAs; false on timeout (uniform across the CTA).
__device__ __forceinline__ bool wait_layer(MlpCtx& c) {
  const bool ok = mbar_wait(c.bar, c.phase);
  c.phase ^= 1u;
  tc_fence_after();
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Epilogue of a hidden layer: acc(row) + bias -> ReLU -> 16-bit -> next A.
template <int N>
__device__ __forceinline__ void hidden_epilogue(const MlpCtx& c, int col, int bias_off, uint8_t* Anext) {
  const int t = threadIdx.x;
  const uint32_t lane = (uint32_t)(t & ~31) << 16;
  const float* bias = reinterpret_cast<const float*>(c.net + kNetImageBias) + bias_off;
#pragma unroll
  for (int c16 = 0; c16 < N / 16; ++c16) {
    uint32_t r[16];
    tmem_ld16(c.tmem + lane + (uint32_t)(col + 16 * c16), r);
    tmem_ld_wait();
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a = fmaxf(__uint_as_float(r[2 * i]) + bias[16 * c16 + 2 * i], 0.0f);
      const float b = fmaxf(__uint_as_float(r[2 * i + 1]) + bias[16 * c16 + 2 * i + 1], 0.0f);
      p[i] = pack2(a, b, c.bf16);
    }
    st_row8(Anext, t, 16 * c16, N, p[0], p[1], p[2], p[3]);
    st_row8(Anext, t, 16 * c16 + 8, N, p[4], p[5], p[6], p[7]);
  }
  tc_fence_before();
  fence_async_smem();
  __syncthreads();
}

// Layers 1..5 for the 128 rows whose layer-1 inputs are in bufY (K = 16).
// Returns false on an MMA timeout.
__device__ bool mlp_tc(MlpCtx& c, float z[4]) {
  if (threadIdx.x == 0) issue_layer(c, c.bufY, 16, kNetImageB1, 64, 0);
  if (!wait_layer(c)) return false;
  hidden_epilogue<64>(c, 0, 0, c.bufX);
  if (threadIdx.x == 0) issue_layer(c, c.bufX, 64, kNetImageB2, 32, 64);
  if (!wait_layer(c)) return false;
  hidden_epilogue<32>(c, 64, 64, c.bufY);
  if (threadIdx.x == 0) issue_layer(c, c.bufY, 32, kNetImageB3, 16, 96);
  if (!wait_layer(c)) return false;
  hidden_epilogue<16>(c, 96, 96, c.bufX);
  if (threadIdx.x == 0) issue_layer(c, c.bufX, 16, kNetImageB4, 16, 112);
  if (!wait_layer(c)) return false;
  hidden_epilogue<16>(c, 112, 112, c.bufY);
  if (threadIdx.x == 0) issue_layer(c, c.bufY, 16, kNetImageB5, 16, 0);
  if (!wait_layer(c)) return false;
  const uint32_t lane = (uint32_t)(threadIdx.x & ~31) << 16;
  uint32_t r[16];
  tmem_ld16(c.tmem + lane, r);
  tmem_ld_wait();
  const float* bias = reinterpret_cast<const float*>(c.net + kNetImageBias) + 128;
#pragma unroll
  for (int k = 0; k < 4; ++k) z[k] = __uint_as_float(r[k]) + bias[k];
  tc_fence_before();
  return true;
}

// Copy the classifier image (16-byte chunks) into shared memory.
__device__ __forceinline__ void load_net_image(uint8_t* dst, const uint8_t* __restrict__ src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < kNetImageBytes / 16; i += blockDim.x) d[i] = s[i];
}

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
  const int t = threadIdx.x;
  load_net_image(s_net, net_image);
  if (t == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  if (t < 32) {
    tmem_alloc(&s_tmem, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  MlpCtx c{s_net, s_bufX, s_bufY, &s_bar, s_tmem, 0u, bf16 != 0};
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
  if (t < 32) tmem_dealloc(s_tmem, 128);
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
  auto put = [&](int off, int N, int K, int n, int k, double w) {
    const uint16_t b = bf16 ? to_bf16_bits(w) : to_fp16_bits(w);
    std::memcpy(img + off + kmajor_offset(n, k, K), &b, 2);
  };
  const int widths[6] = {6, 64, 32, 16, 8, 4};
  const int boff[5] = {kNetImageB1, kNetImageB2, kNetImageB3, kNetImageB4, kNetImageB5};
  const int Kpad[5] = {16, 64, 32, 16, 16};
  const int Npad[5] = {64, 32, 16, 16, 16};
  const int bias_off[5] = {0, 64, 96, 112, 128};
  float* bias = reinterpret_cast<float*>(img + kNetImageBias);
  size_t p = 0;
  for (int l = 0; l < 5; ++l) {
    const int nin = widths[l], nout = widths[l + 1];
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) put(boff[l], Npad[l], Kpad[l], o, i, net.p[p + (size_t)o * nin + i]);
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
