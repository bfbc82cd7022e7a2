// Gradient of the classifier's training loss on the tensor cores: the mean
// binary cross entropy of Eq. (Crossentropy) over the S = 4 sigmoid outputs of
// the 6-64-32-16-8-4 ReLU network of Sec. 3.1, with respect to all 3228
// parameters, for mixed-precision handles (bf16 or fp16 operands, FP32
// accumulation in tensor memory).
//
// Persistent CTAs of 128 threads, two per SM, one 128-sample tile per
// iteration; thread t owns sample row t (MMA row t, TMEM lane t).
//   forward   layers 1-4 by tcgen05.mma exactly as the inference kernel
//             (16-bit activations in TMEM, biases of layers 1-2 on the
//             tensor cores, layer 5 in FP32); every hidden layer's ReLU
//             output is also written, transposed, into shared memory and
//             its ReLU mask kept in registers;
//   deltas    D5 = sigma(z) - y (the 1/(n S) of the mean is applied once, in
//             FP32, to the summed gradient: 16-bit operands then stay in
//             their normal range), D4 and D3 in FP32 on the CUDA cores,
//             D2 = (D3 W3) * relu' and D1 = (D2 W2) * relu' by tcgen05.mma
//             against the transposed weights;
//   gradients dW_l^T (or dW_1) = H_{l-1}^T D_l as tcgen05.mma with K = the
//             tile's 128 samples, accumulated over all of a CTA's tiles in
//             FP32 in tensor memory; a row of ones in each A operand gives
//             the bias gradient sum_s D_l in the same MMA.
// The weight-gradient MMAs run M = 128 rows of which only the first few are
// meaningful: the rows past them read whatever follows in shared memory and
// only fill accumulator rows that are never read.  Per-CTA partial sums go
// to a fixed-order reduction, which applies the 1/(n S).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "mlp_tc.cuh"
#include "tc.cuh"

namespace neno6 {
namespace {

using namespace tc;
using namespace tcmlp;

constexpr int kT = 128;
constexpr uint32_t kSboS = (128 / 8) * 128;  // 8-row group stride of a K = 128 operand
constexpr int kGroup = 2048;                  // bytes of one 8-row group at K = 128
// shared memory (bytes): images, then the weight-gradient A operands (each
// read as 16 groups = 32 KB from its start), then the rest
constexpr int kOffNet = 0;
constexpr int kOffBwd = kOffNet + kNetImageBytes;
constexpr int kOffAH1T = kOffBwd + kBwdImageBytes;  // H1^T (64) + ones (row 64): 9 groups
constexpr int kOffAH2T = kOffAH1T + 9 * kGroup;     // H2^T (32) + ones (row 32): 5 groups
constexpr int kOffAH3T = kOffAH2T + 5 * kGroup;     // H3^T (16) + ones (row 16): 3 groups
constexpr int kOffAH4T = kOffAH3T + 3 * kGroup;     // H4^T (8) + ones (row 8): 2 groups
constexpr int kOffAD1T = kOffAH4T + 2 * kGroup;     // D1^T (64): 8 groups
constexpr int kOffAX0 = kOffAD1T + 8 * kGroup;      // layer-1 input, 128 x 16
constexpr int kOffAD3 = kOffAX0 + 128 * 16 * 2;     // D3, 128 x 16
constexpr int kOffAD2 = kOffAD3 + 128 * 16 * 2;     // D2, 128 x 32
constexpr int kOffBX0T = kOffAD2 + 128 * 32 * 2;    // X0^T (6) + ones (row 6), 16 x 128
constexpr int kOffBD2T = kOffBX0T + 2 * kGroup;     // D2^T, 32 x 128
constexpr int kOffBD3T = kOffBD2T + 4 * kGroup;     // D3^T, 16 x 128
constexpr int kOffBD4T = kOffBD3T + 2 * kGroup;     // D4^T (8), 16 x 128
constexpr int kOffBD5T = kOffBD4T + 2 * kGroup;     // D5^T (4), 16 x 128
constexpr int kOffBar = kOffBD5T + 2 * kGroup;      // mbarrier, TMEM address, timeout flag
constexpr int kOffLoss = kOffBar + 16;              // kT doubles
constexpr int kSmem = ((kOffLoss + kT * 8) + 127) / 128 * 128;
static_assert(kOffAH1T % 128 == 0 && kOffAX0 % 128 == 0, "alignment");
static_assert(kOffAD1T + 16 * kGroup <= kSmem, "the last weight-gradient A operand's 128 rows are addressable");
// two CTAs per SM (2 x 256 TMEM columns)
static_assert(2 * (kSmem + 1024) <= 228 * 1024, "two CTAs per SM");
// TMEM columns: forward / backward working area [0, 64), the weight-gradient
// accumulators from column 128
constexpr uint32_t kAcc1 = 128, kAcc2 = 144, kAcc3 = 176, kAcc4 = 192, kAcc5 = 208;

__device__ __forceinline__ void st_u16(uint8_t* base, uint32_t off, uint16_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(smem_u32(base + off)), "h"(v) : "memory");
}
template <bool BF16>
__device__ __forceinline__ uint16_t bits16(float x) {
  if (BF16) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&b);
  }
  const __half h = __float2half_rn(x);
  return *reinterpret_cast<const uint16_t*>(&h);
}
// Element (row, sample t) of a K = 128 operand (rows x 128 samples).
__device__ __forceinline__ uint32_t kt_off(int row, int t) { return kmajor_offset(row, t, 128); }

// D[col] (+)= A (128 x K rows in smem, group stride sbo) * B (N x K) ^ T,
// K / 16 MMAs issued by this thread; acc0 = accumulate on the first step.
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, const uint8_t* A, uint32_t a_sbo, const uint8_t* B,
                                       uint32_t b_sbo, int K, int N, bool bf16, bool acc0) {
  const uint32_t idesc = idesc_f16(128, N, bf16);
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
  for (int ks = 0; ks < K / 16; ++ks)
    mma_f16(d_tmem, smem_desc(a0 + 256u * ks, 128u, a_sbo), smem_desc(b0 + 256u * ks, 128u, b_sbo), idesc,
            (ks > 0 || acc0) ? 1u : 0u);
}

template <bool BF16>
__global__ void __launch_bounds__(kT, 2) mlp_bwd_tc_kernel(const double* __restrict__ X,
                                                           const uint8_t* __restrict__ y, long long n,
                                                           const uint8_t* __restrict__ net_image,
                                                           const uint8_t* __restrict__ bwd_image,
                                                           float* __restrict__ partial,
                                                           double* __restrict__ partial_loss, int* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* s_net = smem + kOffNet;
  const uint8_t* s_bwd = smem + kOffBwd;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 8);
  int* fail = reinterpret_cast<int*>(smem + kOffBar + 12);
  double* s_loss = reinterpret_cast<double*>(smem + kOffLoss);
  const int t = threadIdx.x;
  const uint32_t lane = (uint32_t)(t & ~31) << 16;

  // images; every operand buffer zeroed, then the constant rows of ones
  for (int i = t; i < kNetImageBytes / 16; i += kT)
    reinterpret_cast<uint4*>(s_net)[i] = reinterpret_cast<const uint4*>(net_image)[i];
  for (int i = t; i < kBwdImageBytes / 16; i += kT)
    reinterpret_cast<uint4*>(smem + kOffBwd)[i] = reinterpret_cast<const uint4*>(bwd_image)[i];
  for (int i = t; i < (kOffBar - kOffAH1T) / 16; i += kT)
    reinterpret_cast<uint4*>(smem + kOffAH1T)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const uint16_t one = bits16<BF16>(1.0f);
  st_u16(smem + kOffAH1T, kt_off(64, t), one);
  st_u16(smem + kOffAH2T, kt_off(32, t), one);
  st_u16(smem + kOffAH3T, kt_off(16, t), one);
  st_u16(smem + kOffAH4T, kt_off(8, t), one);
  st_u16(smem + kOffBX0T, kt_off(6, t), one);
  if (t == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *fail = 0;
  }
  if (t < 32) {
    tmem_alloc(tmem_slot, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  MlpCtx mc{s_net, smem + kOffAX0, bar, tmem, 0u, BF16, fail};
  const float* fbias = reinterpret_cast<const float*>(s_net + kNetImageBias);  // b3 at 0, b4 at 16, b5 at 24
  const float* W4 = reinterpret_cast<const float*>(s_bwd + kBwdW4);          // [8][16]
  const float* W5 = reinterpret_cast<const float*>(s_bwd + kBwdW5);          // [4][8]
  double loss = 0.0;
  const long long tiles = (n + kT - 1) / kT;
  bool first = true;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long s = tile * kT + t;
    const bool live = s < n;
    // ---- Eq. (normalizainput) in FP32
    float x0[6], m = 1.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      x0[j] = live ? (float)X[s * 6 + j] : 0.0f;
      m = fmaxf(m, fabsf(x0[j]));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) x0[j] = x0[j] / m;
    const unsigned lab = live ? y[s] : 0u;
    // the previous tile's weight-gradient MMAs read the operand buffers
    if (!first) wait_layer(mc);
    store_input_row<BF16>(smem + kOffAX0, t, x0);
#pragma unroll
    for (int j = 0; j < 6; ++j) st_u16(smem + kOffBX0T, kt_off(j, t), bits16<BF16>(x0[j]));
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 1 (bias on the ones columns) -> H1
    if (t == 0) issue_layer<BF16>(mc, smem + kOffAX0, 16, kNetImageB1, 64, (int)kColD1);
    wait_layer(mc);
    uint32_t mask1[2] = {0u, 0u};
#pragma unroll
    for (int c32 = 0; c32 < 2; ++c32) {
      uint32_t r[16], q[16];
      tmem_ld16(tmem + lane + kColD1 + 32u * c32, r);
      tmem_ld16(tmem + lane + kColD1 + 32u * c32 + 16u, q);
      tmem_ld_wait();
      uint32_t pk[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float z0 = __uint_as_float(i < 8 ? r[2 * i] : q[2 * i - 16]);
        const float z1 = __uint_as_float(i < 8 ? r[2 * i + 1] : q[2 * i - 15]);
        mask1[c32] |= (z0 > 0.0f ? 1u : 0u) << (2 * i);
        mask1[c32] |= (z1 > 0.0f ? 1u : 0u) << (2 * i + 1);
        pk[i] = relu_pack2<BF16>(z0, z1);
        st_u16(smem + kOffAH1T, kt_off(32 * c32 + 2 * i, t), (uint16_t)(pk[i] & 0xffffu));
        st_u16(smem + kOffAH1T, kt_off(32 * c32 + 2 * i + 1, t), (uint16_t)(pk[i] >> 16));
      }
      tmem_st16(tmem + lane + kColA2 + 16u * c32, pk);
    }
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    // ---- layer 2 (bias K-step on the layer-1 input tile) -> H2
    if (t == 0) issue_layer_t<BF16>(mc, kColA2, 64, kNetImageB2, 32, kColD2, kNetImageB2b);
    wait_layer(mc);
    uint32_t mask2 = 0u;
    {
      uint32_t r[16], q[16];
      tmem_ld16(tmem + lane + kColD2, r);
      tmem_ld16(tmem + lane + kColD2 + 16u, q);
      tmem_ld_wait();
      uint32_t pk[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float z0 = __uint_as_float(i < 8 ? r[2 * i] : q[2 * i - 16]);
        const float z1 = __uint_as_float(i < 8 ? r[2 * i + 1] : q[2 * i - 15]);
        mask2 |= (z0 > 0.0f ? 1u : 0u) << (2 * i);
        mask2 |= (z1 > 0.0f ? 1u : 0u) << (2 * i + 1);
        pk[i] = relu_pack2<BF16>(z0, z1);
        st_u16(smem + kOffAH2T, kt_off(2 * i, t), (uint16_t)(pk[i] & 0xffffu));
        st_u16(smem + kOffAH2T, kt_off(2 * i + 1, t), (uint16_t)(pk[i] >> 16));
      }
      tmem_st16(tmem + lane + kColA3, pk);
    }
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    // ---- layer 3 (+ b3 in FP32) -> H3
    if (t == 0) issue_layer_t<BF16>(mc, kColA3, 32, kNetImageB3, 16, kColD3);
    wait_layer(mc);
    uint32_t mask3 = 0u;
    {
      uint32_t r[16];
      tmem_ld16(tmem + lane + kColD3, r);
      tmem_ld_wait();
      uint32_t pk[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float z0 = __uint_as_float(r[2 * i]) + fbias[2 * i];
        const float z1 = __uint_as_float(r[2 * i + 1]) + fbias[2 * i + 1];
        mask3 |= (z0 > 0.0f ? 1u : 0u) << (2 * i);
        mask3 |= (z1 > 0.0f ? 1u : 0u) << (2 * i + 1);
        pk[i] = relu_pack2<BF16>(z0, z1);
        st_u16(smem + kOffAH3T, kt_off(2 * i, t), (uint16_t)(pk[i] & 0xffffu));
        st_u16(smem + kOffAH3T, kt_off(2 * i + 1, t), (uint16_t)(pk[i] >> 16));
      }
      tmem_st8(tmem + lane + kColA4, pk);
    }
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    // ---- layer 4 (+ b4 in FP32) -> H4; layer 5 in FP32; deltas D5, D4, D3
    if (t == 0) issue_layer_t<BF16>(mc, kColA4, 16, kNetImageB4, 16, kColD4);
    wait_layer(mc);
    float h4[8];
    uint32_t mask4 = 0u;
    {
      uint32_t r[16];
      tmem_ld16(tmem + lane + kColD4, r);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float z = __uint_as_float(r[i]) + fbias[16 + i];
        mask4 |= (z > 0.0f ? 1u : 0u) << i;
        h4[i] = fmaxf(z, 0.0f);
        st_u16(smem + kOffAH4T, kt_off(i, t), bits16<BF16>(h4[i]));
      }
    }
    float d5[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float z = fbias[24 + k];
#pragma unroll
      for (int i = 0; i < 8; ++i) z = fmaf(W5[k * 8 + i], h4[i], z);
      const float yk = (float)((lab >> k) & 1u);
      // -[y log s + (1-y) log(1-s)] = softplus(z) - y z
      if (live) loss += (double)(fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z))) - yk * z);
      d5[k] = live ? 1.0f / (1.0f + __expf(-z)) - yk : 0.0f;
      st_u16(smem + kOffBD5T, kt_off(k, t), bits16<BF16>(d5[k]));
    }
    float d4[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 4; ++k) a = fmaf(W5[k * 8 + i], d5[k], a);
      d4[i] = (mask4 >> i) & 1u ? a : 0.0f;
      st_u16(smem + kOffBD4T, kt_off(i, t), bits16<BF16>(d4[i]));
    }
    float d3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float a = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) a = fmaf(W4[k * 16 + i], d4[k], a);
      d3[i] = (mask3 >> i) & 1u ? a : 0.0f;
      st_u16(smem + kOffBD3T, kt_off(i, t), bits16<BF16>(d3[i]));
    }
    st_row8(smem + kOffAD3, t, 0, 16, pack2<BF16>(d3[0], d3[1]), pack2<BF16>(d3[2], d3[3]),
            pack2<BF16>(d3[4], d3[5]), pack2<BF16>(d3[6], d3[7]));
    st_row8(smem + kOffAD3, t, 8, 16, pack2<BF16>(d3[8], d3[9]), pack2<BF16>(d3[10], d3[11]),
            pack2<BF16>(d3[12], d3[13]), pack2<BF16>(d3[14], d3[15]));
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- D2 = (D3 W3) * relu'(Z2); gradients of layers 5, 4, 3
    if (t == 0) {
      tc_fence_after();
      mma_ss(tmem + 0u, smem + kOffAD3, 256u, s_bwd + kBwdBW3, 256u, 16, 32, BF16, false);
      mma_ss(tmem + kAcc5, smem + kOffAH4T, kSboS, smem + kOffBD5T, kSboS, 128, 16, BF16, !first);
      mma_ss(tmem + kAcc4, smem + kOffAH3T, kSboS, smem + kOffBD4T, kSboS, 128, 16, BF16, !first);
      mma_ss(tmem + kAcc3, smem + kOffAH2T, kSboS, smem + kOffBD3T, kSboS, 128, 16, BF16, !first);
      mma_commit(bar);
    }
    wait_layer(mc);
    {
      uint32_t r[16], q[16];
      tmem_ld16(tmem + lane + 0u, r);
      tmem_ld16(tmem + lane + 16u, q);
      tmem_ld_wait();
      float d2[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float v = __uint_as_float(i < 16 ? r[i] : q[i - 16]);
        d2[i] = (mask2 >> i) & 1u ? v : 0.0f;
        st_u16(smem + kOffBD2T, kt_off(i, t), bits16<BF16>(d2[i]));
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        st_row8(smem + kOffAD2, t, 8 * c, 32, pack2<BF16>(d2[8 * c], d2[8 * c + 1]),
                pack2<BF16>(d2[8 * c + 2], d2[8 * c + 3]), pack2<BF16>(d2[8 * c + 4], d2[8 * c + 5]),
                pack2<BF16>(d2[8 * c + 6], d2[8 * c + 7]));
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- D1 = (D2 W2) * relu'(Z1); gradient of layer 2
    if (t == 0) {
      tc_fence_after();
      mma_ss(tmem + 0u, smem + kOffAD2, 512u, s_bwd + kBwdBW2, 512u, 32, 64, BF16, false);
      mma_ss(tmem + kAcc2, smem + kOffAH1T, kSboS, smem + kOffBD2T, kSboS, 128, 32, BF16, !first);
      mma_commit(bar);
    }
    wait_layer(mc);
#pragma unroll
    for (int c32 = 0; c32 < 2; ++c32) {
      uint32_t r[16], q[16];
      tmem_ld16(tmem + lane + 32u * c32, r);
      tmem_ld16(tmem + lane + 32u * c32 + 16u, q);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float v = __uint_as_float(i < 16 ? r[i] : q[i - 16]);
        st_u16(smem + kOffAD1T, kt_off(32 * c32 + i, t), bits16<BF16>((mask1[c32] >> i) & 1u ? v : 0.0f));
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- gradient of layer 1 (waited for before the next tile's operands)
    if (t == 0) {
      tc_fence_after();
      mma_ss(tmem + kAcc1, smem + kOffAD1T, kSboS, smem + kOffBX0T, kSboS, 128, 16, BF16, !first);
      mma_commit(bar);
    }
    first = false;
    if (__syncthreads_or(*fail)) break;
  }
  if (!first) wait_layer(mc);
  const bool failed = __syncthreads_or(*fail) != 0;
  // ---- this CTA's partial gradients, from the accumulator rows
  float* part = partial + (size_t)blockIdx.x * kNetParams;
  {
    uint32_t r[16];
    tmem_ld16(tmem + lane + kAcc1, r);  // row o of dW1 (o < 64): cols 0..5, db1 in col 6
    tmem_ld_wait();
    if (t < 64) {
#pragma unroll
      for (int i = 0; i < 6; ++i) part[t * 6 + i] = __uint_as_float(r[i]);
      part[384 + t] = __uint_as_float(r[6]);
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {  // row i of dW2^T (i < 64), db2 in row 64
    uint32_t r[16];
    tmem_ld16(tmem + lane + kAcc2 + 16u * c, r);
    tmem_ld_wait();
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      if (t < 64) part[448 + (16 * c + o) * 64 + t] = __uint_as_float(r[o]);
      if (t == 64) part[2496 + 16 * c + o] = __uint_as_float(r[o]);
    }
  }
  {
    uint32_t r[16];
    tmem_ld16(tmem + lane + kAcc3, r);  // row i of dW3^T (i < 32), db3 in row 32
    tmem_ld_wait();
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      if (t < 32) part[2528 + o * 32 + t] = __uint_as_float(r[o]);
      if (t == 32) part[3040 + o] = __uint_as_float(r[o]);
    }
    tmem_ld16(tmem + lane + kAcc4, r);  // row i of dW4^T (i < 16), db4 in row 16
    tmem_ld_wait();
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      if (t < 16) part[3056 + o * 16 + t] = __uint_as_float(r[o]);
      if (t == 16) part[3184 + o] = __uint_as_float(r[o]);
    }
    tmem_ld16(tmem + lane + kAcc5, r);  // row i of dW5^T (i < 8), db5 in row 8
    tmem_ld_wait();
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      if (t < 8) part[3192 + o * 8 + t] = __uint_as_float(r[o]);
      if (t == 8) part[3224 + o] = __uint_as_float(r[o]);
    }
  }
  // block loss (fixed-order tree)
  s_loss[t] = loss;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if (t < w) s_loss[t] += s_loss[t + w];
    __syncthreads();
  }
  if (t == 0) {
    partial_loss[blockIdx.x] = s_loss[0];
    if (failed) atomicOr(status, 4);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (t < 32) tmem_dealloc(tmem, 256);
}

}  // namespace

cudaError_t launch_mlp_bwd_tc(const double* X, const uint8_t* y, long long n, const uint8_t* net_image,
                              const uint8_t* bwd_image, bool bf16, float* grad, float* loss, void* scratch,
                              int* status, cudaStream_t s) {
  const long long tiles = (n + kT - 1) / kT;
  const int blocks = (int)(tiles < 2 * 152 ? tiles : 2 * 152);
  float* partial = static_cast<float*>(scratch);
  double* partial_loss =
      reinterpret_cast<double*>(static_cast<char*>(scratch) + (size_t)blocks * kNetParams * sizeof(float));
  auto kern = bf16 ? mlp_bwd_tc_kernel<true> : mlp_bwd_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kT, kSmem, s>>>(X, y, n, net_image, bwd_image, partial, partial_loss, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_mlp_bwd_reduce(partial, partial_loss, blocks, n, (float)(1.0 / (4.0 * (double)n)), grad, loss, s);
}

}  // namespace neno6
