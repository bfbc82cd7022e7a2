// Mixed-precision NENO6 right-hand side (arXiv 2207.08500, Sec. 4.4 and
// Algorithm 2): every face flux is computed exactly once by a face kernel
// and written to face-flux arrays; a memory-bound FP64 kernel then forms the
// conservative difference and the SSP-RK3 stage update.
//
// Precision split (GB300: the FP64 pipe is ~1/65 of the FP32 pipe, so the
// FP64 work is kept to what the method's conditioning needs):
//   FP64  per-cell Roe inputs (sqrt(rho), u, v, H) and physical fluxes,
//         Roe average and eigenvectors (Sec. 4.4), back-projection, the
//         conservative difference (Eq. (approximateEq)), RK3 accumulation;
//   FP32  LLF alpha, characteristic projection and split, normalisation
//         (Eq. (normalizainput)), candidates, renormalised combination;
//   16-bit tensor cores + FP32 accumulation: the classifier (Sec. 3.1), with
//         rows whose logits fall within +-guard_tau of 0 re-evaluated in FP32
//         on the CUDA cores.
//
// Face kernel: persistent CTAs of one warpgroup (eight per SM, each with 64
// TMEM columns -- all 512 of the SM's -- 64 registers per thread and 26 KB
// of shared memory; the classifier's hidden activations stay in TMEM).  A
// block is 64 faces on 4 grid lines: 4 rows x 16 consecutive x faces, or 4
// columns x 16 consecutive y faces.  Per block:
// stage the 4 x 21 stencil cells (ghost cells by wrap / clamp), compute the
// 64 Roe states once (one thread per face, FP64) while the other half of the
// CTA forms the LLF alpha of every (face, field), then four 128-row
// tensor-core batches of 16 faces x 4 fields x 2 sides.
//
// Reference shift.  A cell near the block's centre is a reference state
// (U_ref, F_ref); every cell is staged as the FP64 difference (U - U_ref,
// F - F_ref) rounded to FP32.  The reconstruction is linear and reproduces
// constants, and the alpha terms of the two sides cancel, so
//   F_face = F_ref + R (g+(delta) + g-(delta))
// exactly: FP32 rounding then acts on the small deviations of the block
// rather than on O(1) fluxes, and the back-projection of the correction can
// run in FP32 while F_ref is added in FP64.  The classifier still sees the
// absolute split fluxes (reference part added back in FP32).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "mlp_tc.cuh"
#include "tc.cuh"

namespace neno6 {
namespace {

using namespace tc;
using namespace tcmlp;

constexpr int kFaces = 64;                     // faces per block
constexpr int kLines = 4;                      // grid lines per block
constexpr int kLineFaces = kFaces / kLines;    // consecutive faces per line
constexpr int kLineCells = kLineFaces + 5;     // stencil cells per line
constexpr int kMaxCells = kLines * kLineCells;  // 84
static_assert(kMaxCells <= 128, "one stencil cell per thread");
// Staged cell c of an x block is (line c / kLineCells, position c % kLineCells);
// of a y block (position c / kLines, line c % kLines).  The reference cell
// sits near the block's centre (line 1, position 10), which keeps the FP32
// deviations small: at most 10 cells along and 2 across the lines.
constexpr int kRefX = 1 * kLineCells + kLineCells / 2;
constexpr int kRefY = (kLineCells / 2) * kLines + 1;
constexpr int kAlign = 128;

constexpr int align_up(int x) { return (x + kAlign - 1) / kAlign * kAlign; }
// dynamic shared-memory layout of the face kernel
constexpr int kOffNet = 0;
// Scratch: during the staging and Roe phase of a block it holds the hand-off
// of 20 cells' FP64 state (1280 B) and, from byte 2048, the FP64 Roe inputs of
// every staged cell (4 x kMaxCells doubles); during the batches the guard
// band's per-warp rows (4 x 128 floats).  The layer-1 input tile is free
// between blocks and holds each cell's FP32 (normal velocity, sound speed).
constexpr int kCellDInScratch = 2048;
constexpr int kScratchBytes = kCellDInScratch + 4 * kMaxCells * 8;
static_assert(kCellDInScratch >= 20 * 64 && kCellDInScratch >= 4 * 128 * 4, "scratch layout");
static_assert(kMaxCells * 8 <= kBufYBytes, "bufY reuse");
constexpr int kOffScratch = align_up(kOffNet + kNetImageBytes);
constexpr int kOffBufY = align_up(kOffScratch + kScratchBytes);
// per cell 8 floats: the (U_n, F_n) deviations, interleaved
constexpr int kOffCellF = align_up(kOffBufY + kBufYBytes);
// rows of L/2 for the fields (u_n - c, entropy, u_n + c): kFaces x 12 floats
// (the shear row of 2D is rebuilt from the Roe velocity); LLF alpha per
// field: kFaces x 4 floats
constexpr int kOffL = align_up(kOffCellF + 8 * kMaxCells * 4);
constexpr int kOffA = align_up(kOffL + kFaces * 12 * 4);
constexpr int kOffR = align_up(kOffA + kFaces * 4 * 4);           // kFaces x 5 floats
constexpr int kOffRef = align_up(kOffR + kFaces * 5 * 4);         // 8 doubles + 8 floats
constexpr int kOffBar = kOffRef + 8 * 8 + 8 * 4;  // mbarrier, TMEM address, timeout flag
constexpr int kOffWtab = align_up(kOffBar + 16);    // 16 masks x 4 renormalised weights
constexpr int kFacesSmem = align_up(kOffWtab + 16 * 4 * 4);
// Eight CTAs per SM: 228 KB of shared memory, allocated in 128-byte units
// plus 1 KB reserved per CTA (and 8 x 64 TMEM columns = 512).
static_assert(kOffBar % 8 == 0 && kFacesSmem % 128 == 0, "alignment");
static_assert(8 * (kFacesSmem + 1024) <= 228 * 1024, "face kernel: CTAs per SM");

// per-cell arrays
enum { CD_S = 0, CD_U = 1, CD_V = 2, CD_H = 3 };

__device__ __forceinline__ int wrap_idx(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// FP64 helpers of the mixed path: hardware reciprocal / reciprocal
// square-root approximations refined by one Newton step (relative error
// ~1e-10 or better).  That is ample here: every Roe quantity is rounded to
// FP32 before use, and an error e|F| in a cell flux enters the FP32
// deviations F - F_ref at ~1e-10 |F|, far below their own rounding; an error
// in the reference flux itself cancels (F_ref + R L (F - F_ref) reproduces a
// constant shift up to the FP32 rounding of R L).
__device__ __forceinline__ double rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt64(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y * y, 1.0);
  return fma(0.5 * y, e, y);
}
// x > 0 (and not NaN) on the integer pipe: the binary64 pattern of a
// positive number (including +inf) is in (0, 0x7ff0000000000000].
__device__ __forceinline__ bool positive64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000ll;
}
// binary64 -> binary32, round to nearest even, on the integer pipe (values
// below the FP32 normal range flush to zero; no overflow in this use).
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e < 897) return __uint_as_float(sign);
  const unsigned long long m = b & 0x000fffffffffffffull;
  const unsigned long long r = m + 0x0fffffffull + ((m >> 29) & 1ull);
  return __uint_as_float(sign | (((unsigned)(e - 896) << 23) + (unsigned)(r >> 29)));
}
// binary32 -> binary64 (exact), on the integer pipe; zero and normal values.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// Warp-cooperative FP32 re-evaluation of the classifier for the rows of this
// warp whose lane has `flagged` set (guard band).  gw: FP32 parameters with
// every W transposed ([in][out]), biases after each W.  ws: 128 floats of
// per-warp shared scratch.
__device__ __forceinline__ void guard_mlp(const float* __restrict__ gw, float* ws, const float (&x)[6],
                                          float (&z)[4], bool flagged) {
  const int lane = threadIdx.x & 31;
  unsigned bal = __ballot_sync(0xffffffffu, flagged);
  while (bal) {
    const int src = __ffs(bal) - 1;
    bal &= bal - 1;
    float xs[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) xs[j] = __shfl_sync(0xffffffffu, x[j], src);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int o = lane + 32 * h;
      float acc = gw[384 + o];
#pragma unroll
      for (int i = 0; i < 6; ++i) acc = fmaf(gw[i * 64 + o], xs[i], acc);
      ws[o] = fmaxf(acc, 0.0f);
    }
    __syncwarp();
    {
      float acc = gw[2496 + lane];
#pragma unroll 8
      for (int i = 0; i < 64; ++i) acc = fmaf(gw[448 + i * 32 + lane], ws[i], acc);
      ws[64 + lane] = fmaxf(acc, 0.0f);
    }
    __syncwarp();
    if (lane < 16) {
      float acc = gw[3040 + lane];
#pragma unroll 8
      for (int i = 0; i < 32; ++i) acc = fmaf(gw[2528 + i * 16 + lane], ws[64 + i], acc);
      ws[96 + lane] = fmaxf(acc, 0.0f);
    }
    __syncwarp();
    if (lane < 8) {
      float acc = gw[3184 + lane];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc = fmaf(gw[3056 + i * 8 + lane], ws[96 + i], acc);
      ws[112 + lane] = fmaxf(acc, 0.0f);
    }
    __syncwarp();
    if (lane < 4) {
      float acc = gw[3224 + lane];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc = fmaf(gw[3192 + i * 4 + lane], ws[112 + i], acc);
      ws[120 + lane] = acc;
    }
    __syncwarp();
    if (lane == src) {
#pragma unroll
      for (int k = 0; k < 4; ++k) z[k] = ws[120 + k];
    }
    __syncwarp();
  }
}

// Geometry of launched block `blk`: the x blocks come first (kLines rows x
// kLineFaces faces), then the y blocks (kLines columns x kLineFaces faces),
// each range starting at its launch offset.
struct BlockGeom {
  int dir;      // 0: x faces, 1: y faces
  int row, f0;  // x block: first row, first face of each line
  int i0, g0;   // y block: first column, first face of each line
};
__device__ __forceinline__ BlockGeom block_geom(long long blk, const FacesMixedArgs& a) {
  BlockGeom b{0, 0, 0, 0, 0};
  if (blk < a.nblk_x) {
    blk += a.blk_x0;
    b.row = (int)(blk / a.bxf) * kLines;
    b.f0 = (int)(blk % a.bxf) * kLineFaces;
  } else {
    const long long q = blk - a.nblk_x + a.blk_y0;
    b.dir = 1;
    b.i0 = (int)(q % a.byc) * kLines;
    b.g0 = (int)(q / a.byc) * kLineFaces;
  }
  return b;
}
// Grid cell (j * nx + i) of staged cell c: ghost cells along the lines by
// periodic wrap or clamp; lines beyond the grid clamp to its last line (their
// faces are not written).
__device__ __forceinline__ size_t staged_cell(const BlockGeom& b, int c, const FacesMixedArgs& a) {
  int gi, gj;
  if (b.dir == 0) {
    gi = wrap_idx(b.f0 - 3 + c % kLineCells, a.nx, a.bcx);
    gj = min(b.row + c / kLineCells, a.ny - 1);
  } else {
    gi = min(b.i0 + c % kLines, a.nx - 1);
    gj = wrap_idx(b.g0 - 3 + c / kLines, a.ny, a.bcy);
  }
  return (size_t)gj * a.nx + gi;
}
// Staged index of face k's first stencil cell (the others follow at stride
// 1 in x blocks, kLines in y blocks).
__device__ __forceinline__ int face_cb0(int dir, int k) {
  return dir == 0 ? (k / kLineFaces) * kLineCells + k % kLineFaces : k;
}
// Face k of the block exists on the grid (x faces 0..nx of rows 0..ny-1,
// y faces 0..ny of columns 0..nx-1).
__device__ __forceinline__ bool face_valid(const BlockGeom& b, int k, int nx, int ny) {
  return b.dir == 0 ? (b.f0 + k % kLineFaces <= nx && b.row + k / kLineFaces < ny)
                    : (b.g0 + k / kLines <= ny && b.i0 + k % kLines < nx);
}

template <int NDIM, bool BF16>
__global__ void __launch_bounds__(kMlpThreads, 8) faces_mixed_kernel(const __grid_constant__ FacesMixedArgs a) {
  constexpr int NV = NDIM == 2 ? 4 : 3;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* s_net = smem + kOffNet;
  double* cd = reinterpret_cast<double*>(smem + kOffScratch + kCellDInScratch);
  float* cf = reinterpret_cast<float*>(smem + kOffCellF);
  float2* cuc = reinterpret_cast<float2*>(smem + kOffBufY);
  float* sL = reinterpret_cast<float*>(smem + kOffL);
  float* sA = reinterpret_cast<float*>(smem + kOffA);
  float* ws = reinterpret_cast<float*>(smem + kOffScratch) + (threadIdx.x >> 5) * 128;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 8);
  int* fail_flag = reinterpret_cast<int*>(smem + kOffBar + 12);
  const int t = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const double gm1 = a.gm1;
  const double hg1 = 0.5 * gm1;
  const float gamma_f = (float)a.gamma;

  for (int i = t; i < kNetImageBytes / 16; i += kMlpThreads)
    reinterpret_cast<uint4*>(s_net)[i] = reinterpret_cast<const uint4*>(a.net_image)[i];
  // weight table in shared memory: lanes index it by their own mask, which a
  // constant-bank read would serialise
  float4* s_wtab = reinterpret_cast<float4*>(smem + kOffWtab);
  if (t < 16) s_wtab[t] = make_float4(a.wtab[t][0], a.wtab[t][1], a.wtab[t][2], a.wtab[t][3]);
  if (t == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *fail_flag = 0;
  }
  if (t < 32) {
    tmem_alloc(tmem_slot, 64);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  MlpCtx mc{s_net, smem + kOffBufY, bar, *tmem_slot, 0u, BF16, fail_flag};
  unsigned long long guarded = 0;
  bool failed = false;

  const long long nblk = a.nblk_x + a.nblk_y;
  double* refd = reinterpret_cast<double*>(smem + kOffRef);      // U_ref[4], F_ref[4] (FP64)
  float* reff = reinterpret_cast<float*>(smem + kOffRef + 64);   // same, FP32
  float* sRf = reinterpret_cast<float*>(smem + kOffR);           // ut, vt, Ht, ct, qt per face
  for (long long blk = blockIdx.x; blk < nblk && !failed; blk += gridDim.x) {
    // ---- block geometry
    const BlockGeom bg = block_geom(blk, a);
    const int dir = bg.dir;
    const int cstride = dir == 0 ? 1 : kLines;
    const int ref_c = dir == 0 ? kRefX : kRefY;
    // thread index rotated by one warp per block, so that the partly
    // occupied cell and Roe phases fall on different warps (and SM
    // sub-partitions) from block to block
    const int tr = (t + (int)((blk & 3) * 32)) & (kMlpThreads - 1);
    // ---- stencil cells (one per thread): FP64 Roe inputs and fluxes
    double U[NV], F[4];
    if (tr < kMaxCells) {
      const size_t g = staged_cell(bg, tr, a);
#pragma unroll
      for (int n = 0; n < NV; ++n) U[n] = a.U[n * plane + g];
      const double rho = U[0], E = U[NV - 1];
      const double rs = rsqrt64(rho);  // 1/sqrt(rho)
      const double rr = rs * rs;       // 1/rho
      const double u = U[1] * rr;
      const double v = NDIM == 2 ? U[2] * rr : 0.0;
      const double rq = NDIM == 2 ? fma(U[2], v, U[1] * u) : U[1] * u;  // rho |u|^2
      const double p = gm1 * fma(-0.5, rq, E);
      const double Ep = E + p;
      if (!positive64(rho) || !positive64(p)) atomicOr(a.status, 1);
      cd[CD_S * kMaxCells + tr] = rho * rs;  // sqrt(rho)
      cd[CD_U * kMaxCells + tr] = u;
      cd[CD_V * kMaxCells + tr] = v;
      cd[CD_H * kMaxCells + tr] = Ep * rr;
      if (NDIM == 1) {
        F[0] = U[1]; F[1] = fma(U[1], u, p); F[2] = Ep * u; F[3] = 0.0;
      } else if (dir == 0) {
        F[0] = U[1]; F[1] = fma(U[1], u, p); F[2] = U[2] * u; F[3] = Ep * u;
      } else {
        F[0] = U[2]; F[1] = U[1] * v; F[2] = fma(U[2], v, p); F[3] = Ep * v;
      }
      cuc[tr] = make_float2(d2f(dir == 0 ? u : v), sqrtf(gamma_f * d2f(p) * d2f(rr)));
      if (tr >= kFaces) {
        // cells kFaces.. are staged by Roe-phase threads: their deviations
        // are formed by the alpha-phase threads, from the scratch
        double* sc = reinterpret_cast<double*>(smem + kOffScratch) + (tr - kFaces) * 8;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          sc[n] = n < NV ? U[n] : 0.0;
          sc[4 + n] = F[n];
        }
      }
      if (tr == ref_c) {  // the block's reference state
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          refd[n] = n < NV ? U[n] : 0.0;
          refd[4 + n] = F[n];
          reff[n] = n < NV ? d2f(U[n]) : 0.0f;
          reff[4 + n] = d2f(F[n]);
        }
      }
    }
    __syncthreads();
    // ---- deviations from the reference, rounded to FP32 (the mass flux is a
    // momentum component: its deviation is that component's)
    auto deviations = [&](int c, const double* Uc, const double* Fc) {
      float w[8];
#pragma unroll
      for (int n = 0; n < 4; ++n) w[2 * n] = n < NV ? d2f(Uc[n] - refd[n]) : 0.0f;
      w[1] = NDIM == 2 && dir == 1 ? w[4] : w[2];
#pragma unroll
      for (int n = 1; n < 4; ++n) w[2 * n + 1] = d2f(Fc[n] - refd[4 + n]);
      float4* dst = reinterpret_cast<float4*>(cf + 8 * c);
      dst[0] = make_float4(w[0], w[1], w[2], w[3]);
      dst[1] = make_float4(w[4], w[5], w[6], w[7]);
    };
    if (tr < kFaces) {
      double Uo[4] = {U[0], U[1], NV > 2 ? U[2] : 0.0, NV > 3 ? U[NV - 1] : 0.0};
      deviations(tr, Uo, F);
      if (tr < kMaxCells - kFaces) {
        const double* sc = reinterpret_cast<const double*>(smem + kOffScratch) + tr * 8;
        deviations(kFaces + tr, sc, sc + 4);
      }
    }
    // ---- Roe average and eigenvectors (FP64), one thread per face; the
    // other half of the CTA forms the LLF alpha of every (face, field)
    const int tq = (tr + 64) & (kMlpThreads - 1);
    if (tq < kFaces) {
      const int k = tq;
      const int cb0 = face_cb0(dir, k);
      const int ca = cb0 + 2 * cstride, cb = cb0 + 3 * cstride;
      const bool valid = face_valid(bg, k, nx, ny);
      const double sa = cd[CD_S * kMaxCells + ca], sb = cd[CD_S * kMaxCells + cb];
      // sqrt(rho)-weighted averages as a + w_b (b - a), w_b = sqrt(rho_b) / (sum)
      const double wb = sb * rcp64(sa + sb);
      const double ua = cd[CD_U * kMaxCells + ca], va = cd[CD_V * kMaxCells + ca], Ha = cd[CD_H * kMaxCells + ca];
      const double ut = fma(wb, cd[CD_U * kMaxCells + cb] - ua, ua);
      const double vt = fma(wb, cd[CD_V * kMaxCells + cb] - va, va);
      const double Ht = fma(wb, cd[CD_H * kMaxCells + cb] - Ha, Ha);
      const double qt = fma(vt, vt, ut * ut);
      const double hq = 0.5 * qt;
      const double c2 = gm1 * (Ht - hq);
      if (valid && !positive64(c2)) atomicOr(a.status, 2);
      const double ic = rsqrt64(c2);  // 1/c
      const double ct = c2 * ic;
      // rows of L = R^-1 in halves: hb1 = b1/2 = (gamma-1)/(2c^2), hb2 = b2/2 =
      // hb1 |u|^2/2, hic = 1/(2c).  L/2 is stored (the split's factor 1/2,
      // exact in binary): its entries are these halves rounded to FP32 and
      // scaled by exact powers of 2.
      const double hb1 = hg1 * (ic * ic);
      const double hb2 = hb1 * hq;
      const double hic = 0.5 * ic;
      const double hnc = (dir == 0 ? ut : vt) * hic;
      const double hb1u = hb1 * ut, hb1v = hb1 * vt;
      const double hbn = dir == 0 ? hb1u : hb1v;
      const double sn = hbn + hic, dn = hic - hbn;  // (b1 u_n + 1/c)/2, (1/c - b1 u_n)/2
      const float fb1u = d2f(hb1u), fb1v = d2f(hb1v), fb1 = d2f(hb1);
      const float l0 = d2f(hb2 + hnc), l4 = d2f(fma(-2.0, hb2, 1.0)), l12 = d2f(hb2 - hnc);
      const float fsn = d2f(sn), fdn = d2f(dn);
      // three stored rows: the u_n - c, entropy and u_n + c fields
      float4* L = reinterpret_cast<float4*>(sL + k * 12);
      const float h = 0.5f;
      if (NDIM == 1) {
        L[0] = make_float4(h * l0, -h * fsn, h * fb1, 0.f);
        L[1] = make_float4(h * l4, fb1u, -fb1, 0.f);
        L[2] = make_float4(h * l12, h * fdn, h * fb1, 0.f);
      } else {
        L[0] = make_float4(h * l0, dir == 0 ? -h * fsn : -h * fb1u, dir == 0 ? -h * fb1v : -h * fsn, h * fb1);
        L[1] = make_float4(h * l4, fb1u, fb1v, -fb1);
        L[2] = make_float4(h * l12, dir == 0 ? h * fdn : -h * fb1u, dir == 0 ? -h * fb1v : h * fdn, h * fb1);
      }
      float* R = sRf + k * 5;
      R[0] = d2f(ut); R[1] = d2f(vt); R[2] = d2f(Ht); R[3] = d2f(ct); R[4] = d2f(qt);
    } else {
      // LLF alpha per field: max over the six stencil cells of |u_n - c|,
      // |u_n| and |u_n + c|
      const int k = tq - kFaces;
      const int cb0 = face_cb0(dir, k);
      float am = 0.0f, a0 = 0.0f, ap = 0.0f;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float2 uc = cuc[cb0 + j * cstride];
        am = fmaxf(am, fabsf(uc.x - uc.y));
        a0 = fmaxf(a0, fabsf(uc.x));
        ap = fmaxf(ap, fabsf(uc.x + uc.y));
      }
      reinterpret_cast<float4*>(sA)[k] = NDIM == 2 ? make_float4(am, a0, a0, ap) : make_float4(am, a0, ap, 0.0f);
    }
    __syncthreads();
    // ---- four tensor-core batches of 16 faces x 4 fields x 2 sides
    for (int mt = 0; mt < kFaces / 16; ++mt) {
      const int k = mt * 16 + (t >> 3);
      const int fld = (t >> 1) & 3;
      const int m = min(fld, NV - 1);
      const int side = t & 1;
      const int cb0 = face_cb0(dir, k);
      const bool valid = fld < NV && face_valid(bg, k, nx, ny);
      // row m of L/2; the shear row of 2D is (-u_t, e_t) / 2
      float4 Lv;
      if (NDIM == 2 && m == 2) {
        const float tt = sRf[k * 5 + (dir == 0 ? 1 : 0)];
        Lv = make_float4(-0.5f * tt, dir == 0 ? 0.0f : 0.5f, dir == 0 ? 0.5f : 0.0f, 0.0f);
      } else {
        Lv = reinterpret_cast<const float4*>(sL + k * 12)[m == 0 ? 0 : (m == NV - 1 ? 2 : 1)];
      }
      const float Lr[4] = {Lv.x, Lv.y, Lv.z, Lv.w};
      const float alpha = sA[k * 4 + m];
      const float sgn_alpha = side ? -alpha : alpha;
      // reference part of this side's split flux: (L F_ref +- alpha L U_ref)/2
      float vr = Lr[0] * reff[0], gr = Lr[0] * reff[4];
#pragma unroll
      for (int n = 1; n < NV; ++n) {
        vr = fmaf(Lr[n], reff[n], vr);
        gr = fmaf(Lr[n], reff[4 + n], gr);
      }
      const float cref = fmaf(sgn_alpha, vr, gr);
      // deviations of the split flux from the reference part, in this side's
      // stencil order ("+" side cells i-2..i+3, "-" side the mirror image
      // i+3..i-2).  Both sides of a (face, field), adjacent lanes, project the
      // same six cells: each lane projects the first three cells of its own
      // order and takes the other three, (v, g) pairs, from its partner.
      float ds[6];
      float2 vg[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        // (v, g) = L_m/2 . (U_j, F_j) deviations, both in one packed FMA chain
        const int j = side ? 5 - q : q;
        const float4* src = reinterpret_cast<const float4*>(cf + 8 * (cb0 + j * cstride));
        const float4 p0 = src[0], p1 = src[1];
        vg[q] = __fmul2_rn(make_float2(Lr[0], Lr[0]), make_float2(p0.x, p0.y));
        vg[q] = __ffma2_rn(make_float2(Lr[1], Lr[1]), make_float2(p0.z, p0.w), vg[q]);
        vg[q] = __ffma2_rn(make_float2(Lr[2], Lr[2]), make_float2(p1.x, p1.y), vg[q]);
        if (NV == 4) vg[q] = __ffma2_rn(make_float2(Lr[3], Lr[3]), make_float2(p1.z, p1.w), vg[q]);
        ds[q] = fmaf(sgn_alpha, vg[q].x, vg[q].y);
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        // the partner's q-th cell is this side's (5 - q)-th
        const float v = __shfl_xor_sync(0xffffffffu, vg[q].x, 1);
        const float g = __shfl_xor_sync(0xffffffffu, vg[q].y, 1);
        ds[5 - q] = fmaf(sgn_alpha, v, g);
      }
      float mx = 1.0f, s[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        s[j] = cref + ds[j];
        mx = fmaxf(mx, fabsf(s[j]));
      }
      // mx >= 1: the approximate reciprocal (within 1 ulp) is ample for an
      // input that is rounded to 16 bits next
      float inv;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(mx));
      float x[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) x[j] = s[j] * inv;
      unsigned eta;
      if (a.mask_mode == kMaskMLP) {
        store_input_row<BF16>(mc.bufY, t, x);
        fence_async_smem();
        __syncthreads();
        float z[4];
        if (!mlp_tc<BF16>(mc, z)) {
          failed = true;
          break;
        }
        if (a.guard_tau > 0.0f) {
          bool flag = false;
#pragma unroll
          for (int q = 0; q < 4; ++q) flag |= fabsf(z[q]) < a.guard_tau;
          guarded += (flag && valid) ? 1 : 0;
          guard_mlp(a.guard_w, ws, x, z, flag);
        }
        eta = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) eta |= (z[q] > 0.0f ? 1u : 0u) << q;
      } else {
        eta = a.mask_mode == kMaskRough ? 15u : 0u;
      }
      // candidates and renormalised combination of the deviations (FP32);
      // first-order fallback
      float gsum;
      if (eta == 15u) {
        gsum = ds[2];
      } else {
        float f[4];
        f[0] = fmaf(a.cand[0][2], ds[3], fmaf(a.cand[0][1], ds[2], a.cand[0][0] * ds[1]));
        f[1] = fmaf(a.cand[1][2], ds[4], fmaf(a.cand[1][1], ds[3], a.cand[1][0] * ds[2]));
        f[2] = fmaf(a.cand[2][2], ds[2], fmaf(a.cand[2][1], ds[1], a.cand[2][0] * ds[0]));
        f[3] = fmaf(a.cand[3][3], ds[5], fmaf(a.cand[3][2], ds[4], fmaf(a.cand[3][1], ds[3], a.cand[3][0] * ds[2])));
        // discarded stencils have weight 0 in the table (fma(0, f, g) = g)
        const float4 w = s_wtab[eta];
        gsum = fmaf(w.w, f[3], fmaf(w.z, f[2], fmaf(w.y, f[1], w.x * f[0])));
      }
      const float gh = gsum + __shfl_xor_sync(0xffffffffu, gsum, 1);
      const unsigned eta_other = __shfl_xor_sync(0xffffffffu, eta, 1);
      float ghq[4];
      const int fb = (t & 31) & ~7;
#pragma unroll
      for (int q = 0; q < 4; ++q) ghq[q] = __shfl_sync(0xffffffffu, gh, fb + 2 * q);
      if (side == 0 && valid) {
        // back-projection of the correction (FP32), plus F_ref (FP64)
        const float* Rd = sRf + k * 5;
        const float ut = Rd[0], vt = Rd[1], Ht = Rd[2], ct = Rd[3], qt = Rd[4];
        const float nt = dir == 0 ? ut : vt;
        const float ntc = nt * ct;
        // row n of R against the waves (u_n - c, entropy, [shear,] u_n + c)
        // is (A - B, C, [D,] A + B), selected without branches:
        //   density (1, 0, 1, 0); energy (H, u_n c, |u|^2/2, u_t);
        //   normal momentum (u_n, c, u_n, 0); tangential (u_t, 0, u_t, 1)
        const int n = m;
        const float tt = dir == 0 ? vt : ut;
        const bool is_rho = n == 0, is_e = n == NV - 1, is_nrm = n == 1 + dir;
        const float A = is_rho ? 1.0f : (is_e ? Ht : (is_nrm ? nt : tt));
        const float B = is_e ? ntc : (is_nrm ? ct : 0.0f);
        const float C = is_rho ? 1.0f : (is_e ? 0.5f * qt : (is_nrm ? nt : tt));
        float corr = (A - B) * ghq[0];
        corr = fmaf(C, ghq[1], corr);
        if (NDIM == 2) {
          const float D = is_e ? tt : ((is_rho || is_nrm) ? 0.0f : 1.0f);
          corr = fmaf(D, ghq[2], corr);
          corr = fmaf(A + B, ghq[3], corr);
        } else {
          corr = fmaf(A + B, ghq[2], corr);
        }
        const double Fh = refd[4 + n] + f2d(corr);
        size_t idx;
        if (dir == 0) {
          const int f = bg.f0 + k % kLineFaces, r = bg.row + k / kLineFaces;
          idx = ((size_t)n * ny + r) * (nx + 1) + f;
          a.Fx[idx] = Fh;
        } else {
          const int g = bg.g0 + k / kLines, i = bg.i0 + k % kLines;
          idx = ((size_t)n * (ny + 1) + g) * nx + i;
          a.Fy[idx] = Fh;
          idx += (size_t)NV * ny * (nx + 1);
        }
        if (a.mask_out) a.mask_out[idx] = (uint8_t)(eta | (eta_other << 4));
      }
      __syncthreads();
    }
    __syncthreads();
  }
  if (failed && t == 0) atomicOr(a.status, 4);
  if (a.guard_count && guarded) atomicAdd(a.guard_count, guarded);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (t < 32) tmem_dealloc(*tmem_slot, 64);
}

// Conservative difference (FP64) and optional SSP-RK3 stage update of the
// rows j0 .. j1 - 1: thread per cell, a 2D grid of rows (blockIdx.y,
// grid-stride beyond 65535 rows) by runs of 256 cells.  The difference of each direction is one DADD and the
// two directions combine in one DMUL + DFMA: 4 FP64 operations per field.
template <int NDIM>
__global__ void __launch_bounds__(256) diff_mixed_kernel(DiffArgs a) {
  constexpr int NV = NDIM == 2 ? 4 : 3;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double dt = a.stage ? *a.dt_dev : 0.0;
  if (a.stage == 3 && a.t_dev && i == 0 && blockIdx.y == 0) *a.t_dev = *a.t_dev + dt;
  if (i >= a.nx) return;
  const size_t plane = (size_t)a.nx * a.ny;
  // with periodic boundaries faces 0 and nx (ny) are one physical face: both
  // neighbours use face 0's value, so the difference telescopes exactly
  const int ir = (i + 1 == a.nx && a.bcx == 0) ? 0 : i + 1;
  for (int j = a.j0 + (int)blockIdx.y; j < a.j1; j += gridDim.y) {
    const int jr = (j + 1 == a.ny && a.bcy == 0) ? 0 : j + 1;
    const size_t cell = (size_t)j * a.nx + i;
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      const double* fx = a.Fx + ((size_t)n * a.ny + j) * (a.nx + 1);
      const double rx = -a.inv_dx * (fx[ir] - fx[i]);
      double r = rx;
      if (NDIM == 2) {
        const double* fy = a.Fy + (size_t)n * (a.ny + 1) * a.nx + i;
        r = fma(-a.inv_dy, fy[(size_t)jr * a.nx] - fy[(size_t)j * a.nx], rx);
      }
      const size_t e = n * plane + cell;
      double val = r;
      if (a.stage == 1) val = fma(dt, r, a.U[e]);
      else if (a.stage == 2) val = fma(0.75, a.U0[e], 0.25 * fma(dt, r, a.U[e]));
      else if (a.stage == 3) val = fma(a.third, a.U0[e], a.two_thirds * fma(dt, r, a.U[e]));
      a.out[e] = val;
    }
  }
}

// Largest wave speeds max(|u|+c), max(|v|+c) of the mixed path's step (Sec.
// 4.4's CFL condition): the pressure, whose difference E - rho|u|^2/2 cancels
// at high Mach numbers, in FP64 (reciprocal of rho by the hardware
// approximation and one Newton step); velocities and sound speed in FP32.
// The step size only has to respect the CFL bound, and a relative error of
// ~1e-7 in it changes nothing else: the RK3 accumulation stays FP64.  The
// maxima are handed to dt_kernel as binary64 bit patterns, like the FP64
// path's (non-negative values order like their patterns).
template <int NDIM>
__global__ void __launch_bounds__(256) cfl_mixed_kernel(const double* __restrict__ U, int nx, int ny,
                                                        size_t k0, size_t k1, double gamma,
                                                        unsigned long long* smax, int* status) {
  const size_t plane = (size_t)nx * ny;
  const double gm1 = gamma - 1.0;
  const float gamma_f = (float)gamma;
  float mx = 0.0f, my = 0.0f;
  bool bad = false;
  for (size_t k = k0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < k1;
       k += (size_t)gridDim.x * blockDim.x) {
    const double rho = U[k];
    const double m = U[plane + k];
    const double n = NDIM == 2 ? U[2 * plane + k] : 0.0;
    const double E = U[(NDIM == 2 ? 3 : 2) * plane + k];
    const double rr = rcp64(rho);
    const double p = gm1 * fma(-0.5 * rr, fma(n, n, m * m), E);
    bad |= !positive64(rho) || !positive64(p);
    const float rf = d2f(rr);
    const float c = sqrtf(gamma_f * d2f(p) * rf);
    mx = fmaxf(mx, fabsf(d2f(m) * rf) + c);
    if (NDIM == 2) my = fmaxf(my, fabsf(d2f(n) * rf) + c);
  }
  if (bad) atomicOr(status, 1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&smax[0], (unsigned long long)__double_as_longlong(f2d(mx)));
    if (NDIM == 2) atomicMax(&smax[1], (unsigned long long)__double_as_longlong(f2d(my)));
  }
}

// dt = cfl / (max(|u|+c)/dx + max(|v|+c)/dy), clipped to t_end (one thread).
__global__ void dt_kernel(const unsigned long long* smax, int ndim, double dx, double dy, double cfl,
                          double t_end, const double* t_dev, double* dt_dev, double* dt_user) {
  double s = __longlong_as_double((long long)smax[0]) / dx;
  if (ndim == 2) s = s + __longlong_as_double((long long)smax[1]) / dy;
  double dt = cfl / s;
  const double t = *t_dev;
  if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
  *dt_dev = dt;
  if (dt_user) *dt_user = dt;
}

}  // namespace

void build_guard_image(const NetF64& net, float* g) {
  const int widths[6] = {6, 64, 32, 16, 8, 4};
  size_t p = 0;
  for (int l = 0; l < 5; ++l) {
    const int nin = widths[l], nout = widths[l + 1];
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) g[p + (size_t)i * nout + o] = (float)net.p[p + (size_t)o * nin + i];
    p += (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) g[p + o] = (float)net.p[p + o];
    p += nout;
  }
}

cudaError_t launch_faces_mixed(int ndim, FacesMixedArgs& a, cudaStream_t s, int row0, int row1) {
  // x blocks: nx + 1 faces per row in runs of kLineFaces, rows in groups of
  // kLines; y blocks: columns in groups of kLines, ny + 1 faces per column
  // in runs of kLineFaces.  Rows row0 .. row1 - 1: their row groups, and the
  // runs of y faces from row0 up to row1 (the last run when row1 == ny).
  a.bxf = (a.nx + 1 + kLineFaces - 1) / kLineFaces;
  a.byc = (a.nx + kLines - 1) / kLines;
  const int rg0 = row0 / kLines;
  const int rg1 = row1 == a.ny ? (a.ny + kLines - 1) / kLines : row1 / kLines;
  const int fr0 = row0 / kLineFaces;
  const int fr1 = row1 == a.ny ? (a.ny + 1 + kLineFaces - 1) / kLineFaces : row1 / kLineFaces;
  a.blk_x0 = (long long)a.bxf * rg0;
  a.nblk_x = (long long)a.bxf * (rg1 - rg0);
  a.blk_y0 = (long long)a.byc * fr0;
  a.nblk_y = ndim == 2 ? (long long)a.byc * (fr1 - fr0) : 0;
  const long long nblk = a.nblk_x + a.nblk_y;
  if (nblk <= 0) return cudaSuccess;
  // persistent grid: eight resident CTAs per SM (registers, shared memory,
  // 64 TMEM columns each)
  const int blocks = (int)(nblk < 152 * 8 ? nblk : 152 * 8);
  auto kern = ndim == 2 ? (a.bf16 ? faces_mixed_kernel<2, true> : faces_mixed_kernel<2, false>)
                        : (a.bf16 ? faces_mixed_kernel<1, true> : faces_mixed_kernel<1, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kFacesSmem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kMlpThreads, kFacesSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diff_mixed(int ndim, const DiffArgs& a, cudaStream_t s) {
  const int rows = a.j1 - a.j0;
  if (rows <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((a.nx + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
  if (ndim == 2) diff_mixed_kernel<2><<<grid, 256, 0, s>>>(a);
  else diff_mixed_kernel<1><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_cfl_mixed(int ndim, const double* U, int nx, int ny, double gamma, unsigned long long* smax,
                             int* status, cudaStream_t s, int row0, int row1, bool zero) {
  if (zero) {
    cudaError_t e = cudaMemsetAsync(smax, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  const size_t k0 = (size_t)row0 * nx, k1 = (size_t)row1 * nx;
  if (k1 <= k0) return cudaSuccess;
  unsigned blocks = (unsigned)((k1 - k0 + 255) / 256);
  if (blocks > 152u * 8u) blocks = 152u * 8u;
  if (ndim == 2) cfl_mixed_kernel<2><<<blocks, 256, 0, s>>>(U, nx, ny, k0, k1, gamma, smax, status);
  else cfl_mixed_kernel<1><<<blocks, 256, 0, s>>>(U, nx, ny, k0, k1, gamma, smax, status);
  return cudaGetLastError();
}

cudaError_t launch_dt(const unsigned long long* smax, int ndim, double dx, double dy, double cfl, double t_end,
                      const double* t_dev, double* dt_dev, double* dt_user, cudaStream_t s) {
  dt_kernel<<<1, 1, 0, s>>>(smax, ndim, dx, dy, cfl, t_end, t_dev, dt_dev, dt_user);
  return cudaGetLastError();
}

}  // namespace neno6
