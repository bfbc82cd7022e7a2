// Classifier training on the GPU (Sec. 3.3, Table 2): mini-batch Adam
// (Kingma & Ba, Algorithm 1: beta1 0.9, beta2 0.999, epsilon 1e-8) on the
// mean binary cross entropy of Eq. (Crossentropy), the batches taken in the
// order of a caller-given permutation of the samples.
//
// Mini-batch Adam is sequential (every step reads the parameters the
// previous step wrote), so one persistent cluster of CTAs runs all the steps
// of a call, sharing each step's batch (below).  A CTA's four warps share the
// forward and backward pass of its samples (lane = sample, each layer's
// outputs split among the warps; mlp_fb.cuh) against the parameters in
// shared memory.  No launch per step and no global-memory round trip of the
// parameters; the gradient and the loss are reduced in a fixed order, so a
// call is deterministic.
#include "internal.h"
#include "mlp_fb.cuh"

namespace neno6 {
namespace {

using namespace mlpfb;

// The training loop on a cluster of kCl CTAs (kCl SMs): every step's
// batch is shared among the CTAs (at most kPerCta samples each).  Each CTA
// runs its samples' forward and backward passes and forms the partial
// gradient of all 3228 parameters over them; after a cluster barrier, CTA r
// sums the partials of the parameter slice it owns over the kCl CTAs (read
// from their shared memory, in rank order: deterministic), applies Adam to
// that slice (its moments stay in its shared memory for the whole call) and
// publishes the new values; after a second barrier every CTA gathers the
// slices into its copy of the parameters.
constexpr int kCl = 8;
constexpr int kCT = 128;                                    // threads per CTA
constexpr int kPerCta = (kMaxTrainBatch + kCl - 1) / kCl;    // samples per CTA (24)
constexpr int kCPitch = kPerCta + 1;
constexpr int kSlice = (kNetParams + kCl - 1) / kCl;         // 404 parameters per CTA
constexpr int kCPer = (kNetParams + kCT - 1) / kCT;          // partial sums per thread
// floats: W, staging (kRows rows, then a row of ones), partial gradient,
// published slice, Adam m and v
constexpr int kCOffW = 0, kCOffSt = kNetParams, kCOffOnes = kCOffSt + kRows * kCPitch;
constexpr int kCOffPart = kCOffOnes + kCPitch;
constexpr int kCOffSlice = kCOffPart + kNetParams, kCOffM = kCOffSlice + kSlice, kCOffV = kCOffM + kSlice;
constexpr int kCSmemFloats = kCOffV + kSlice;
static_assert(kPerCta <= 32 && kSlice <= 4 * kCT, "one warp of samples, four slice entries per thread");

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// float at shared-memory pointer p of the cluster's CTA `rank`
__device__ __forceinline__ float ld_cluster(const float* p, uint32_t rank) {
  uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p)), remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
  return v;
}

__global__ void __launch_bounds__(kCT, 1) mlp_train_cluster_kernel(const MlpTrainArgs a) {
  extern __shared__ float sm[];
  float* W = sm + kCOffW;
  float* st = sm + kCOffSt;
  float* ones = sm + kCOffOnes;
  float* part = sm + kCOffPart;
  float* slice = sm + kCOffSlice;
  float* mm = sm + kCOffM;
  float* vv = sm + kCOffV;
  __shared__ double sl[kCT];
  const int t = threadIdx.x;
  const uint32_t rank = cluster_rank();
  const int p_lo = (int)rank * kSlice;
  for (int i = t; i < kNetParams; i += kCT) W[i] = a.params[i];
  for (int i = t; i < kCPitch; i += kCT) ones[i] = 1.0f;
  for (int i = t; i < kSlice; i += kCT) {
    const int p = p_lo + i;
    mm[i] = p < kNetParams ? a.m[p] : 0.0f;
    vv[i] = p < kNetParams ? a.v[p] : 0.0f;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float lr = a.lr;
  double loss_sum = 0.0;
  bool bad_index = false;
  double p1 = pow(0.9, (double)a.t0), p2 = pow(0.999, (double)a.t0);
  __syncthreads();
  const long long steps = (a.n_perm + a.batch - 1) / a.batch;
  for (long long step = 0; step < steps; ++step) {
    const long long s0 = step * a.batch;
    const int nb = (int)min((long long)a.batch, a.n_perm - s0);
    const int per = (nb + kCl - 1) / kCl;
    const int first = min((int)rank * per, nb), ns = min(per, nb - first);
    // ---- this CTA's samples: forward and backward, lane = sample, the four
    // warps sharing every layer's outputs
    {
      const int lane = t & 31, warp = t >> 5;
      const bool active = lane < kPerCta;  // lanes past kPerCta have no staged column
      bool live = lane < ns;
      long long idx = 0;
      if (live) {
        idx = a.perm[s0 + first + lane];
        if (idx < 0 || idx >= a.n) {
          if (warp == 0) bad_index = true;
          live = false;
          idx = 0;
        }
      }
      float xr[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) xr[j] = live ? (float)a.X[idx * 6 + j] : 0.0f;
      double loss = 0.0;
      sample_fwd_bwd_coop<kCPitch, kCT / 32>(W, st, active ? lane : 0, warp, active, live, xr,
                                             live ? a.y[idx] : 0u, 1.0f / (4.0f * (float)nb), loss);
      if (warp == 0 && lane < kPerCta) loss_sum += loss * (0.25 / (double)nb);
    }
    // ---- partial gradient of every parameter over these samples, four
    // parameters per pass over the samples
#pragma unroll 1
    for (int q = 0; q < kCPer; q += 4) {
      float g4[4];
      param_grads<kCPitch, 4>(st, ones, t + q * kCT, kCT, ns, g4);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = t + (q + u) * kCT;
        if (p < kNetParams) part[p] = g4[u];
      }
    }
    cluster_sync();
    // ---- this CTA's slice: sum over the CTAs (rank order), Adam, publish
    p1 *= 0.9;
    p2 *= 0.999;
    const float c1 = (float)(1.0 / (1.0 - p1));
    const float c2 = (float)(1.0 / (1.0 - p2));
    for (int i = t; i < kSlice; i += kCT) {
      const int p = p_lo + i;
      if (p < kNetParams) {
        float g = 0.0f;
#pragma unroll
        for (int r = 0; r < kCl; ++r) g += ld_cluster(part + p, (uint32_t)r);
        mm[i] = fmaf(b1, mm[i], (1.0f - b1) * g);
        vv[i] = fmaf(b2, vv[i], (1.0f - b2) * (g * g));
        const float mh = mm[i] * c1, vh = vv[i] * c2;
        slice[i] = W[p] - lr * mh / (sqrtf(vh) + eps);
      }
    }
    cluster_sync();
    // ---- every CTA gathers the new parameters
    for (int p = t; p < kNetParams; p += kCT) {
      const int owner = p / kSlice;
      W[p] = ld_cluster(slice + (p - owner * kSlice), (uint32_t)owner);
    }
    __syncthreads();
  }
  // results: every CTA holds the parameters; each writes its own slice and
  // moments
  for (int i = t; i < kSlice; i += kCT) {
    const int p = p_lo + i;
    if (p < kNetParams) {
      a.params[p] = W[p];
      a.m[p] = mm[i];
      a.v[p] = vv[i];
    }
  }
  // loss: per CTA a fixed-order tree, then the CTAs in rank order
  sl[t] = loss_sum;
  __syncthreads();
  for (int w = kCT / 2; w > 0; w >>= 1) {
    if (t < w) sl[t] += sl[t + w];
    __syncthreads();
  }
  float* lossf = part;  // the CTA's loss as two floats (hi, lo) for the gather
  if (t == 0) {
    const double v = sl[0];
    lossf[0] = (float)v;
    lossf[1] = (float)(v - (double)(float)v);
  }
  cluster_sync();
  if (rank == 0 && t == 0 && a.loss_sum) {
    double tot = 0.0;
    for (int r = 0; r < kCl; ++r) tot += (double)ld_cluster(lossf, (uint32_t)r) + (double)ld_cluster(lossf + 1, (uint32_t)r);
    *a.loss_sum = tot;
  }
  if (bad_index) atomicOr(a.status, 8);
  cluster_sync();  // no CTA leaves while another may still read its memory
}

}  // namespace

cudaError_t launch_mlp_train(const MlpTrainArgs& a, cudaStream_t s) {
  // one cluster of kCl CTAs
  const size_t smem = (size_t)kCSmemFloats * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(mlp_train_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCl, 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, mlp_train_cluster_kernel, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace neno6
