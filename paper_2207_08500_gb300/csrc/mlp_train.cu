// Classifier training on the GPU (Sec. 3.3, Table 2): mini-batch Adam
// (Kingma & Ba, Algorithm 1: beta1 0.9, beta2 0.999, epsilon 1e-8) on the
// mean binary cross entropy of Eq. (Crossentropy), the batches taken in the
// order of a caller-given permutation of the samples.
//
// Mini-batch Adam is sequential (every step reads the parameters the
// previous step wrote), so one persistent CTA of 192 threads runs all the
// steps of a call: per step one thread per sample runs the forward and
// backward pass (mlp_fb.cuh) against the parameters in shared memory, then
// each thread sums the batch gradient of the ~17 parameters it owns and
// applies the Adam update to them, keeping their moments in registers.  No
// launch per step and no global-memory round trip of the parameters; each
// thread accumulates its samples' share of the loss and the shares are
// reduced in a fixed order at the end, so a call is deterministic.
#include "internal.h"
#include "mlp_fb.cuh"

namespace neno6 {
namespace {

using namespace mlpfb;

constexpr int kB = kMaxTrainBatch;      // threads = largest batch
constexpr int kPitch = kB + 1;          // feature-major rows, padded
constexpr int kPer = (kNetParams + kB - 1) / kB;  // parameters owned per thread
constexpr int kSmemFloats = kNetParams + kRows * kPitch;
constexpr int kRed = 256;  // loss reduction width (power of two >= kB)
static_assert(kSmemFloats * 4 + kRed * 8 <= 227 * 1024, "training kernel shared memory");

__global__ void __launch_bounds__(kB, 1) mlp_train_kernel(const MlpTrainArgs a) {
  extern __shared__ float sm[];
  float* W = sm;
  float* st = sm + kNetParams;
  __shared__ double sl[kRed];
  const int t = threadIdx.x;
  for (int i = t; i < kNetParams; i += kB) W[i] = a.params[i];
  float mq[kPer], vq[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int p = t + q * kB;
    mq[q] = p < kNetParams ? a.m[p] : 0.0f;
    vq[q] = p < kNetParams ? a.v[p] : 0.0f;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float lr = a.lr;
  double loss_sum = 0.0;  // this thread's samples' share of sum_steps (batch-mean BCE)
  bool bad_index = false;
  // beta^t of the step before this call's first (bias corrections)
  double p1 = pow(0.9, (double)a.t0), p2 = pow(0.999, (double)a.t0);
  __syncthreads();
  const long long steps = (a.n_perm + a.batch - 1) / a.batch;
  for (long long step = 0; step < steps; ++step) {
    const long long s0 = step * a.batch;
    const int nb = (int)min((long long)a.batch, a.n_perm - s0);
    bool live = t < nb;
    long long idx = 0;
    if (live) {
      idx = a.perm[s0 + t];
      if (idx < 0 || idx >= a.n) {  // out-of-range sample: skipped, reported
        bad_index = true;
        live = false;
        idx = 0;
      }
    }
    float xr[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) xr[j] = live ? (float)a.X[idx * 6 + j] : 0.0f;
    double loss = 0.0;
    sample_fwd_bwd<kPitch>(W, st, t, live, xr, live ? a.y[idx] : 0u, 1.0f / (4.0f * (float)nb), loss);
    loss_sum += loss * (0.25 / (double)nb);
    __syncthreads();
    // Adam (Kingma & Ba, Algorithm 1) on the owned parameters; the step count
    // runs on across calls (t0 steps before this one)
    p1 *= 0.9;
    p2 *= 0.999;
    const float c1 = (float)(1.0 / (1.0 - p1));  // 1 / (1 - beta1^t)
    const float c2 = (float)(1.0 / (1.0 - p2));  // 1 / (1 - beta2^t)
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int p = t + q * kB;
      if (p < kNetParams) {
        const float g = param_grad<kPitch>(st, p, nb);
        mq[q] = fmaf(b1, mq[q], (1.0f - b1) * g);
        vq[q] = fmaf(b2, vq[q], (1.0f - b2) * (g * g));
        const float mh = mq[q] * c1, vh = vq[q] * c2;
        W[p] -= lr * mh / (sqrtf(vh) + eps);
      }
    }
    __syncthreads();
  }
  for (int i = t; i < kNetParams; i += kB) a.params[i] = W[i];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int p = t + q * kB;
    if (p < kNetParams) {
      a.m[p] = mq[q];
      a.v[p] = vq[q];
    }
  }
  // sum of the per-step batch-mean losses: fixed-order tree over the threads
  sl[t] = loss_sum;
  if (t < kRed - kB) sl[kB + t] = 0.0;
  __syncthreads();
  for (int w = kRed / 2; w > 0; w >>= 1) {
    if (t < w) sl[t] += sl[t + w];
    __syncthreads();
  }
  if (t == 0 && a.loss_sum) *a.loss_sum = sl[0];
  if (bad_index) atomicOr(a.status, 8);
}

}  // namespace

cudaError_t launch_mlp_train(const MlpTrainArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)kSmemFloats * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_train_kernel<<<1, kB, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace neno6
