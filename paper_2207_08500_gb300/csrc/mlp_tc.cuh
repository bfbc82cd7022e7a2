// Tensor-core MLP shared by the mixed-precision kernels (see mixed.cu for the
// scheme): one warpgroup of 128 threads, thread t = MMA row t = TMEM lane t.
// Layer 1 reads its input tile from shared memory; layers 2-4 read their
// input (the previous layer's ReLU output rounded to 16 bits) from tensor
// memory, written there by the epilogue into columns the previous layer's
// accumulator has vacated.  64 TMEM columns:
//   layer 1 D [0,64) -> A2 [0,32) (64 values, two per column)
//   layer 2 D [32,64) -> A3 [0,16);  layer 3 D [16,32) -> A4 [32,40);
//   layer 4 D [48,64).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "tc.cuh"

namespace neno6 {
namespace tcmlp {

using namespace tc;

constexpr int kMlpThreads = 128;
constexpr int kBufYBytes = 128 * 16 * 2;  // A1 (K = 16): the layer-1 input tile
constexpr uint32_t kColD1 = 0, kColA2 = 0, kColD2 = 32, kColA3 = 0, kColD3 = 16, kColA4 = 32, kColD4 = 48;

// Round two FP32 values to bf16/fp16 and pack them, a in bits 0-15.
template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if (BF16) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// ReLU, round to the nearest finite 16-bit value and pack (a in bits 0-15):
// one cvt instruction per pair.  Saturating to the largest finite value keeps
// fp16 activations finite.
template <bool BF16>
__device__ __forceinline__ uint32_t relu_pack2(float a, float b) {
  uint32_t d;
  if (BF16)
    asm("cvt.rn.relu.satfinite.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  else
    asm("cvt.rn.relu.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
  return d;
}

// The 16-bit pair (1, 1) and (1, 0): the constant columns of the layer-1
// input row that carry the biases of layers 1 and 2.
template <bool BF16>
__device__ __forceinline__ constexpr uint32_t ones2() { return BF16 ? 0x3F803F80u : 0x3C003C00u; }
template <bool BF16>
__device__ __forceinline__ constexpr uint32_t one0() { return BF16 ? 0x00003F80u : 0x00003C00u; }

// Store 8 consecutive K values (one core-matrix row) of row `row`.
__device__ __forceinline__ void st_row8(uint8_t* base, int row, int k0, int K, uint32_t a, uint32_t b,
                                        uint32_t c, uint32_t d) {
  const uint32_t addr = smem_u32(base + kmajor_offset(row, k0, K));
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// Row `row` of the layer-1 input tile (K = 16): the six normalised stencil
// values in columns 0-5 and, in bf16, again in 6-11 (against W1's hi and lo
// terms), then 1, 1, 1 in columns ones_col(BF16) .. + 2 (bias terms), zeros.
template <bool BF16>
__device__ __forceinline__ void store_input_row(uint8_t* bufY, int row, const float x[6]) {
  const uint32_t p01 = pack2<BF16>(x[0], x[1]), p23 = pack2<BF16>(x[2], x[3]), p45 = pack2<BF16>(x[4], x[5]);
  if (BF16) {
    static_assert(ones_col(true) == 12, "bf16: ones occupy columns 12-14");
    st_row8(bufY, row, 0, 16, p01, p23, p45, p01);
    st_row8(bufY, row, 8, 16, p23, p45, ones2<BF16>(), one0<BF16>());
  } else {
    static_assert(ones_col(false) == 6, "fp16: ones occupy columns 6-8");
    st_row8(bufY, row, 0, 16, p01, p23, p45, ones2<BF16>());
    st_row8(bufY, row, 8, 16, one0<BF16>(), 0u, 0u, 0u);
  }
}

struct MlpCtx {
  const uint8_t* net;  // shared-memory image (kNetImage* layout)
  uint8_t* bufY;       // layer-1 input tile
  uint64_t* bar;
  uint32_t tmem;
  uint32_t phase;
  bool bf16;
  int* fail;           // shared timeout flag
};

// Issue one layer (thread 0): K/16 MMAs of K = 16 into TMEM column `col`,
// plus, if Bb_off >= 0, a bias K-step (the layer-1 input tile in bufY, whose
// columns ones_col .. ones_col + 2 hold 1, times the bias tile at Bb_off).
template <bool BF16>
__device__ __forceinline__ void issue_layer(const MlpCtx& c, const uint8_t* A, int K, int B_off, int N,
                                            int col, int Bb_off = -1) {
  const uint32_t sbo = (uint32_t)(K / 8) * 128u;
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(c.net + B_off);
  const uint32_t idesc = idesc_f16(128, N, BF16);
  tc_fence_after();
  for (int ks = 0; ks < K / 16; ++ks)
    mma_f16(c.tmem + (uint32_t)col, smem_desc(a0 + 256u * ks, 128u, sbo),
            smem_desc(b0 + 256u * ks, 128u, sbo), idesc, ks > 0 ? 1u : 0u);
  if (Bb_off >= 0)
    mma_f16(c.tmem + (uint32_t)col, smem_desc(smem_u32(c.bufY), 128u, 256u),
            smem_desc(smem_u32(c.net + Bb_off), 128u, 256u), idesc, 1u);
  mma_commit(c.bar);
}

// Issue one layer (thread 0) whose input sits in tensor memory at column
// colA: K/16 MMAs of K = 16 into column colD, plus, if Bb_off >= 0, the bias
// K-step on the layer-1 input tile in bufY.
template <bool BF16>
__device__ __forceinline__ void issue_layer_t(const MlpCtx& c, uint32_t colA, int K, int B_off, int N,
                                              uint32_t colD, int Bb_off = -1) {
  const uint32_t sbo = (uint32_t)(K / 8) * 128u;
  const uint32_t b0 = smem_u32(c.net + B_off);
  const uint32_t idesc = idesc_f16(128, N, BF16);
  tc_fence_after();
  for (int ks = 0; ks < K / 16; ++ks)
    mma_f16_ta(c.tmem + colD, c.tmem + colA + 8u * ks, smem_desc(b0 + 256u * ks, 128u, sbo), idesc,
               ks > 0 ? 1u : 0u);
  if (Bb_off >= 0)
    mma_f16(c.tmem + colD, smem_desc(smem_u32(c.bufY), 128u, 256u),
            smem_desc(smem_u32(c.net + Bb_off), 128u, 256u), idesc, 1u);
  mma_commit(c.bar);
}

// Wait for the layer's MMAs (bounded).  A timeout is recorded in the shared
// flag *fail and acted on, uniformly, at the end of the chain.
__device__ __forceinline__ void wait_layer(MlpCtx& c) {
  if (!mbar_wait(c.bar, c.phase)) *c.fail = 1;
  c.phase ^= 1u;
  tc_fence_after();
}

// Epilogue of a hidden tensor-core layer (bias already accumulated): this
// row of the FP32 accumulator at colD -> ReLU -> 16-bit pairs -> this row of
// the next layer's operand at colA in tensor memory (32 values per round
// trip).  colA may overlap colD: each 32-value chunk is read before the
// packed 16 columns are written, and chunk q writes below chunk q+1.
template <int N, bool BF16>
__device__ __forceinline__ void hidden_epilogue(const MlpCtx& c, uint32_t colD, uint32_t colA) {
  const int t = threadIdx.x;
  const uint32_t lane = (uint32_t)(t & ~31) << 16;
#pragma unroll
  for (int c32 = 0; c32 < N / 32; ++c32) {
    uint32_t r[16], s[16];
    tmem_ld16(c.tmem + lane + colD + 32u * c32, r);
    tmem_ld16(c.tmem + lane + colD + 32u * c32 + 16u, s);
    tmem_ld_wait();
    uint32_t p[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      p[i] = relu_pack2<BF16>(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
      p[8 + i] = relu_pack2<BF16>(__uint_as_float(s[2 * i]), __uint_as_float(s[2 * i + 1]));
    }
    tmem_st16(c.tmem + lane + colA + 16u * c32, p);
  }
  tmem_st_wait();
  tc_fence_before();
  __syncthreads();
}

// Layer 3's accumulator row (TMEM columns kColD3..) + b3 -> ReLU -> 16-bit ->
// this row of layer 4's operand (8 TMEM columns at kColA4); layer 4 on the
// tensor cores (N = 16, rows 8-15 of B4 zero) into columns kColD4..; its row
// + b4 -> ReLU, then layer 5 (8 -> 4) in FP32 on the CUDA cores, two outputs
// per packed FMA (each output accumulates over its inputs in order, one
// rounding per FMA).
template <bool BF16>
__device__ __forceinline__ void tail_layers(MlpCtx& c, float z[4]) {
  const int t = threadIdx.x;
  const uint32_t lane = (uint32_t)(t & ~31) << 16;
  const float* bias = reinterpret_cast<const float*>(c.net + kNetImageBias);
  uint32_t r[16];
  tmem_ld16(c.tmem + lane + kColD3, r);
  tmem_ld_wait();
  uint32_t p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 b = reinterpret_cast<const float2*>(bias)[i];
    const float2 h = __fadd2_rn(make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1])), b);
    p[i] = relu_pack2<BF16>(h.x, h.y);
  }
  tmem_st8(c.tmem + lane + kColA4, p);
  tmem_st_wait();
  tc_fence_before();
  __syncthreads();
  if (t == 0) issue_layer_t<BF16>(c, kColA4, 16, kNetImageB4, 16, kColD4);
  wait_layer(c);
  tmem_ld16(c.tmem + lane + kColD4, r);
  tmem_ld_wait();
  tc_fence_before();
  const float2* W5t = reinterpret_cast<const float2*>(c.net + kNetImageW5);  // [8][2] pairs
  float h4[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) h4[o] = fmaxf(__uint_as_float(r[o]) + bias[16 + o], 0.0f);
  float2 a5[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) a5[k] = reinterpret_cast<const float2*>(bias + 24)[k];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 h = make_float2(h4[i], h4[i]);
#pragma unroll
    for (int k = 0; k < 2; ++k) a5[k] = __ffma2_rn(W5t[i * 2 + k], h, a5[k]);
  }
  z[0] = a5[0].x;
  z[1] = a5[0].y;
  z[2] = a5[1].x;
  z[3] = a5[1].y;
}

// The classifier for the 128 rows whose layer-1 inputs are in bufY (K = 16,
// written by store_input_row): layers 1-4 on the tensor cores, layer 5 on the
// CUDA cores, TMEM columns as listed at the top.  Every epilogue ends with its
// TMEM stores waited, a fence and a barrier before the next issue, so each
// layer's MMAs see their whole operand and never overwrite columns a thread
// is still reading.  Returns false (uniformly) if an MMA wait timed out.
template <bool BF16>
__device__ __forceinline__ bool mlp_tc(MlpCtx& c, float z[4]) {
  if (threadIdx.x == 0) issue_layer<BF16>(c, c.bufY, 16, kNetImageB1, 64, (int)kColD1);
  wait_layer(c);
  hidden_epilogue<64, BF16>(c, kColD1, kColA2);
  // layer 2 also reads the input tile in bufY (its bias K-step)
  if (threadIdx.x == 0) issue_layer_t<BF16>(c, kColA2, 64, kNetImageB2, 32, kColD2, kNetImageB2b);
  wait_layer(c);
  hidden_epilogue<32, BF16>(c, kColD2, kColA3);
  if (threadIdx.x == 0) issue_layer_t<BF16>(c, kColA3, 32, kNetImageB3, 16, kColD3);
  wait_layer(c);
  tail_layers<BF16>(c, z);
  // every thread's timeout record is visible after this barrier
  return __syncthreads_or(*c.fail) == 0;
}

// The 6-32-32-32-4 network of the width study (neno6_classify only), image
// layout kNarrow*: layers 1-3 on the tensor cores (N = 32), every
// accumulator in TMEM columns [0,32) and every 16-bit operand of layers 2-3
// in [32,48); b1 and b2 ride on the ones columns as above, b3 is added in
// FP32 and layer 4 (32 -> 4) runs in FP32 on the CUDA cores on the FP32
// ReLU output of layer 3 (bias, then an FMA per input in ascending order).
template <bool BF16>
__device__ __forceinline__ bool mlp_tc_narrow(MlpCtx& c, float z[4]) {
  const int t = threadIdx.x;
  if (t == 0) issue_layer<BF16>(c, c.bufY, 16, kNarrowB1, 32, 0);
  wait_layer(c);
  hidden_epilogue<32, BF16>(c, 0, 32);
  if (t == 0) issue_layer_t<BF16>(c, 32, 32, kNarrowB2, 32, 0, kNarrowB2b);
  wait_layer(c);
  hidden_epilogue<32, BF16>(c, 0, 32);
  if (t == 0) issue_layer_t<BF16>(c, 32, 32, kNarrowB3, 32, 0);
  wait_layer(c);
  const uint32_t lane = (uint32_t)(t & ~31) << 16;
  uint32_t r[16], q[16];
  tmem_ld16(c.tmem + lane, r);
  tmem_ld16(c.tmem + lane + 16u, q);
  tmem_ld_wait();
  tc_fence_before();
  const float* b3 = reinterpret_cast<const float*>(c.net + kNarrowBias3);
  const float* w4t = reinterpret_cast<const float*>(c.net + kNarrowW4);  // [32][4], then b4
#pragma unroll
  for (int k = 0; k < 4; ++k) z[k] = w4t[128 + k];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const float h = fmaxf(__uint_as_float(i < 16 ? r[i] : q[i - 16]) + b3[i], 0.0f);
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = fmaf(w4t[i * 4 + k], h, z[k]);
  }
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
