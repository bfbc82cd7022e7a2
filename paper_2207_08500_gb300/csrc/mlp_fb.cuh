// Per-sample forward and backward pass of the classifier's training loss,
// shared by the gradient kernel (mlp_bwd.cu) and the training kernel
// (mlp_train.cu).  The network is the 6-64-32-16-8-4 ReLU MLP of Sec. 3.1,
// the loss the mean binary cross entropy of Eq. (Crossentropy) over the S = 4
// sigmoid outputs, all in FP32.
//
// One thread per sample.  The weights W (weights-file order: per layer
// W[out][in] then b[out]) are broadcast from shared memory; every layer's
// input and every delta are staged feature-major in shared memory, column
// `col` of rows of length PITCH, for the parameter-gradient sums that follow.
#pragma once

#include <cmath>

#include "internal.h"

namespace neno6 {
namespace mlpfb {

// parameter offsets and layer widths
__host__ __device__ constexpr int wofs(int l) { return l == 0 ? 0 : l == 1 ? 448 : l == 2 ? 2528 : l == 3 ? 3056 : 3192; }
__host__ __device__ constexpr int wid(int l) { return l == 0 ? 6 : l == 1 ? 64 : l == 2 ? 32 : l == 3 ? 16 : l == 4 ? 8 : 4; }
// staged rows: inputs x0 (6) x1 (64) x2 (32) x3 (16) x4 (8); deltas d1..d5
constexpr int kX0 = 0, kX1 = 6, kX2 = 70, kX3 = 102, kX4 = 118;
constexpr int kD1 = 126, kD2 = 190, kD3 = 222, kD4 = 238, kD5 = 246, kRows = 250;

__device__ __forceinline__ float softplus(float z) {  // log(1 + e^z), stable
  return fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z)));
}

// Forward and backward pass of one sample (raw stencil x, label bits lab;
// `live` false stages zeros).  inv_nS = 1 / (4 n) for a batch of n samples.
// Adds the sample's BCE sum over the four outputs to `loss`.
template <int PITCH>
__device__ __forceinline__ void sample_fwd_bwd(const float* W, float* st, int col, bool live, const float (&xr)[6],
                                               unsigned lab, float inv_nS, double& loss) {
  // ---- forward (Eq. (normalizainput), (reconstuction), (activationfunction))
  float x0[6], m = 1.0f;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    x0[j] = live ? xr[j] : 0.0f;
    m = fmaxf(m, fabsf(x0[j]));
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    x0[j] = x0[j] / m;
    st[(kX0 + j) * PITCH + col] = x0[j];
  }
  float h1[64];
#pragma unroll
  for (int o = 0; o < 64; ++o) {
    float a = W[wofs(0) + 384 + o];
#pragma unroll
    for (int i = 0; i < 6; ++i) a = fmaf(W[wofs(0) + o * 6 + i], x0[i], a);
    h1[o] = fmaxf(a, 0.0f);
    st[(kX1 + o) * PITCH + col] = h1[o];
  }
  float h2[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float a = W[wofs(1) + 2048 + o];
#pragma unroll
    for (int i = 0; i < 64; ++i) a = fmaf(W[wofs(1) + o * 64 + i], h1[i], a);
    h2[o] = fmaxf(a, 0.0f);
    st[(kX2 + o) * PITCH + col] = h2[o];
  }
  float h3[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) {
    float a = W[wofs(2) + 512 + o];
#pragma unroll
    for (int i = 0; i < 32; ++i) a = fmaf(W[wofs(2) + o * 32 + i], h2[i], a);
    h3[o] = fmaxf(a, 0.0f);
    st[(kX3 + o) * PITCH + col] = h3[o];
  }
  float h4[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    float a = W[wofs(3) + 128 + o];
#pragma unroll
    for (int i = 0; i < 16; ++i) a = fmaf(W[wofs(3) + o * 16 + i], h3[i], a);
    h4[o] = fmaxf(a, 0.0f);
    st[(kX4 + o) * PITCH + col] = h4[o];
  }
  // ---- output: loss and dL/dz = (sigma(z) - y) / (n S); ReLU masks of the
  // backward pass are re-read from the staged activations (fewer live
  // registers)
  asm volatile("" ::: "memory");
  float d5[4];
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
    st[(kD5 + k) * PITCH + col] = d5[k];
  }
  // ---- backward: delta_l = (W_{l+1}^T delta_{l+1}) * relu'(pre-activation)
  float d4[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) a = fmaf(W[wofs(4) + k * 8 + i], d5[k], a);
    d4[i] = st[(kX4 + i) * PITCH + col] > 0.0f ? a : 0.0f;
    st[(kD4 + i) * PITCH + col] = d4[i];
  }
  float d3[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) a = fmaf(W[wofs(3) + k * 16 + i], d4[k], a);
    d3[i] = st[(kX3 + i) * PITCH + col] > 0.0f ? a : 0.0f;
    st[(kD3 + i) * PITCH + col] = d3[i];
  }
  float d2[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) a = fmaf(W[wofs(2) + k * 32 + i], d3[k], a);
    d2[i] = st[(kX2 + i) * PITCH + col] > 0.0f ? a : 0.0f;
    st[(kD2 + i) * PITCH + col] = d2[i];
  }
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) a = fmaf(W[wofs(1) + k * 64 + i], d2[k], a);
    st[(kD1 + i) * PITCH + col] = st[(kX1 + i) * PITCH + col] > 0.0f ? a : 0.0f;
  }
}

// The same forward and backward pass, the CTA's NW warps cooperating on up
// to 32 samples (lane = sample = staged column `col`): every layer's outputs
// are split among the warps (output o to warp o % NW), each output computed
// exactly as above -- its bias (or 0), then an fma chain over its inputs in
// ascending order, the inputs read back from the staged rows -- with a CTA
// barrier between layers; warp 0 forms the outputs, the loss and dL/dz.  The
// staged rows are therefore bit for bit those of sample_fwd_bwd, in a
// quarter of its latency with four warps.  Every thread of the CTA must call
// it: lanes with `active` false (no staged column) only meet the barriers,
// active lanes past the batch pass `live` false.
template <int PITCH, int NW, int kG = 8>
__device__ __forceinline__ void sample_fwd_bwd_coop(const float* W, float* st, int col, int warp, bool active,
                                                    bool live, const float (&xr)[6], unsigned lab, float inv_nS,
                                                    double& loss) {
  if (warp == 0 && active) {
    float x0[6], m = 1.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      x0[j] = live ? xr[j] : 0.0f;
      m = fmaxf(m, fabsf(x0[j]));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) st[(kX0 + j) * PITCH + col] = x0[j] / m;
  }
  __syncthreads();
  // hidden layers l = 0..3: input rows xin, output rows xout
#pragma unroll 1
  for (int l = 0; l < 4; ++l) {
    const int nin = wid(l), nout = wid(l + 1);
    const int xin = l == 0 ? kX0 : l == 1 ? kX1 : l == 2 ? kX2 : kX3;
    const int xout = l == 0 ? kX1 : l == 1 ? kX2 : l == 2 ? kX3 : kX4;
    const float* Wl = W + wofs(l);
    // kG of this warp's outputs at a time (o0, o0 + NW, ...), independent
    // chains over one pass of the inputs
#pragma unroll 1
    for (int o0 = warp; active && o0 < nout; o0 += NW * kG) {
      float a[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) a[g] = o0 + g * NW < nout ? Wl[nout * nin + o0 + g * NW] : 0.0f;
      for (int i = 0; i < nin; ++i) {
        const float xv = st[(xin + i) * PITCH + col];
#pragma unroll
        for (int g = 0; g < kG; ++g)
          if (o0 + g * NW < nout) a[g] = fmaf(Wl[(o0 + g * NW) * nin + i], xv, a[g]);
      }
#pragma unroll
      for (int g = 0; g < kG; ++g)
        if (o0 + g * NW < nout) st[(xout + o0 + g * NW) * PITCH + col] = fmaxf(a[g], 0.0f);
    }
    __syncthreads();
  }
  if (warp == 0 && active) {  // output layer, loss and dL/dz
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float z = W[wofs(4) + 32 + k];
#pragma unroll
      for (int i = 0; i < 8; ++i) z = fmaf(W[wofs(4) + k * 8 + i], st[(kX4 + i) * PITCH + col], z);
      const float yk = (float)((lab >> k) & 1u);
      const float sig = 1.0f / (1.0f + __expf(-z));
      if (live) loss += (double)(softplus(z) - yk * z);
      st[(kD5 + k) * PITCH + col] = live ? (sig - yk) * inv_nS : 0.0f;
    }
  }
  __syncthreads();
  // backward l = 3..0: delta of layer l's output from the delta above it
#pragma unroll 1
  for (int l = 3; l >= 0; --l) {
    const int nin = wid(l + 1), nup = wid(l + 2);  // this delta's width, the one above
    const int dup = l == 3 ? kD5 : l == 2 ? kD4 : l == 1 ? kD3 : kD2;
    const int dout = l == 3 ? kD4 : l == 2 ? kD3 : l == 1 ? kD2 : kD1;
    const int xact = l == 3 ? kX4 : l == 2 ? kX3 : l == 1 ? kX2 : kX1;
    const float* Wu = W + wofs(l + 1);  // W_{l+2}[nup][nin]
#pragma unroll 1
    for (int i0 = warp; active && i0 < nin; i0 += NW * kG) {
      float a[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) a[g] = 0.0f;
      for (int k = 0; k < nup; ++k) {
        const float dv = st[(dup + k) * PITCH + col];
#pragma unroll
        for (int g = 0; g < kG; ++g)
          if (i0 + g * NW < nin) a[g] = fmaf(Wu[k * nin + i0 + g * NW], dv, a[g]);
      }
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const int i = i0 + g * NW;
        if (i < nin) st[(dout + i) * PITCH + col] = st[(xact + i) * PITCH + col] > 0.0f ? a[g] : 0.0f;
      }
    }
    __syncthreads();
  }
}

// Gradients of the NP parameters p0, p0 + stride, ... summed over the first
// `ns` staged samples -- dW = sum delta x (x the layer's input), db = sum
// delta, each an fma chain over the samples in ascending order -- as
// independent chains in one pass over the samples and without branches: a
// bias gradient is an fma against `ones` (a staged row of 1.0f), which rounds
// as the plain sum does.  Parameters past kNetParams produce values the
// caller drops.
template <int PITCH, int NP>
__device__ __forceinline__ void param_grads(const float* st, const float* ones, int p0, int stride, int ns,
                                            float (&out)[NP]) {
  const float* dp[NP];
  const float* xp[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int p = min(p0 + q * stride, kNetParams - 1);
    int l = 4;
    while (l > 0 && p < wofs(l)) --l;
    const int nin = wid(l), nout = wid(l + 1);
    const int r = p - wofs(l);
    const int drow = (l == 0 ? kD1 : l == 1 ? kD2 : l == 2 ? kD3 : l == 3 ? kD4 : kD5);
    const int xrow = (l == 0 ? kX0 : l == 1 ? kX1 : l == 2 ? kX2 : l == 3 ? kX3 : kX4);
    const bool isw = r < nout * nin;
    dp[q] = st + (drow + (isw ? r / nin : r - nout * nin)) * PITCH;
    xp[q] = isw ? st + (xrow + r % nin) * PITCH : ones;
    out[q] = 0.0f;
  }
  for (int j = 0; j < ns; ++j) {
#pragma unroll
    for (int q = 0; q < NP; ++q) out[q] = fmaf(dp[q][j], xp[q][j], out[q]);
  }
}

}  // namespace mlpfb
}  // namespace neno6
