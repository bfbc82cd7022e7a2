// Tensor-core MLP shared by the mixed-precision kernels (see mixed.cu for the
// scheme): one warpgroup of 128 threads, thread t = MMA row t = TMEM lane t.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "tc.cuh"

namespace neno6 {
namespace tcmlp {

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
  int* fail;           // shared timeout flag
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

// Wait for the layer's MMAs (bounded).  A timeout is recorded in the shared
// flag *fail and acted on, uniformly, at the end of the chain.
__device__ __forceinline__ void wait_layer(MlpCtx& c) {
  if (!mbar_wait(c.bar, c.phase)) *c.fail = 1;
  c.phase ^= 1u;
  tc_fence_after();
}

// Epilogue of a hidden tensor-core layer: acc(row) + bias -> ReLU -> 16-bit
// -> this row of the next layer's operand.
template <int N>
__device__ __forceinline__ void hidden_epilogue(const MlpCtx& c, int col, int bias_off, uint8_t* Anext) {
  const int t = threadIdx.x;
  const uint32_t lane = (uint32_t)(t & ~31) << 16;
  const float* bias = reinterpret_cast<const float*>(c.net + kNetImageBias) + bias_off;
  // fp16 activations are kept below the fp16 maximum
  const float hi = c.bf16 ? 3.0e38f : 65000.0f;
#pragma unroll
  for (int c16 = 0; c16 < N / 16; ++c16) {
    uint32_t r[16];
    tmem_ld16(c.tmem + lane + (uint32_t)(col + 16 * c16), r);
    tmem_ld_wait();
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a = fminf(fmaxf(__uint_as_float(r[2 * i]) + bias[16 * c16 + 2 * i], 0.0f), hi);
      const float b = fminf(fmaxf(__uint_as_float(r[2 * i + 1]) + bias[16 * c16 + 2 * i + 1], 0.0f), hi);
      p[i] = pack2(a, b, c.bf16);
    }
    st_row8(Anext, t, 16 * c16, N, p[0], p[1], p[2], p[3]);
    st_row8(Anext, t, 16 * c16 + 8, N, p[4], p[5], p[6], p[7]);
  }
  tc_fence_before();
  fence_async_smem();
  __syncthreads();
}

// Layer 3's accumulator row (TMEM column col) + bias -> ReLU, then layers
// 4-5 (16 -> 8 -> 4) in FP32 on the CUDA cores.
__device__ __forceinline__ void tail_layers(const MlpCtx& c, int col, float z[4]) {
  const uint32_t lane = (uint32_t)(threadIdx.x & ~31) << 16;
  uint32_t r[16];
  tmem_ld16(c.tmem + lane + (uint32_t)col, r);
  tmem_ld_wait();
  tc_fence_before();
  const float* bias = reinterpret_cast<const float*>(c.net + kNetImageBias);
  const float* W4 = reinterpret_cast<const float*>(c.net + kNetImageW4);
  const float* W5 = reinterpret_cast<const float*>(c.net + kNetImageW5);
  float h3[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) h3[i] = fmaxf(__uint_as_float(r[i]) + bias[96 + i], 0.0f);
  float h4[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    float a = bias[112 + o];
#pragma unroll
    for (int i = 0; i < 16; ++i) a = fmaf(W4[o * 16 + i], h3[i], a);
    h4[o] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float a = bias[120 + k];
#pragma unroll
    for (int i = 0; i < 8; ++i) a = fmaf(W5[k * 8 + i], h4[i], a);
    z[k] = a;
  }
}

// The classifier for the 128 rows whose layer-1 inputs are in bufY (K = 16):
// layers 1-3 on the tensor cores, layers 4-5 on the CUDA cores.  64 TMEM
// columns: layer 1 -> [0,64); layer 2 -> [0,32) once layer 1's epilogue has
// read its columns (the epilogue ends with a fence and a barrier before the
// next issue); layer 3 -> [32,48).  Returns false (uniformly) if an MMA wait
// timed out.
__device__ __forceinline__ bool mlp_tc(MlpCtx& c, float z[4]) {
  if (threadIdx.x == 0) issue_layer(c, c.bufY, 16, kNetImageB1, 64, 0);
  wait_layer(c);
  hidden_epilogue<64>(c, 0, 0, c.bufX);
  if (threadIdx.x == 0) issue_layer(c, c.bufX, 64, kNetImageB2, 32, 0);
  wait_layer(c);
  hidden_epilogue<32>(c, 0, 64, c.bufY);
  if (threadIdx.x == 0) issue_layer(c, c.bufY, 32, kNetImageB3, 16, 32);
  wait_layer(c);
  tail_layers(c, 32, z);
  // every thread's timeout record is visible after this barrier
  return __syncthreads_or(*c.fail) == 0;
}

// Copy the classifier image (16-byte chunks) into shared memory.
__device__ __forceinline__ void load_net_image(uint8_t* dst, const uint8_t* __restrict__ src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < kNetImageBytes / 16; i += blockDim.x) d[i] = s[i];
}

}  // namespace tcmlp
}  // namespace neno6
