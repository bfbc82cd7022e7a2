// Scalar conservation laws u_t + f(u)_x = 0 on a 1D grid with the same
// NENO6 reconstruction (Sec. 4.1 linear advection, f = u; Sec. 4.2 Burgers,
// f = u^2 / 2), FP64.  Local Lax-Friedrichs split with alpha = max over the
// six stencil cells of |f'(u)|, the "-" side mirrored about the face, the
// classifier of Sec. 3.1 on each side's normalised split fluxes (Eq.
// (normalizainput)), the candidates and renormalised weights of Algorithm 2,
// the conservative difference of Eq. (approximateEq) and SSP-RK3.
//
// One thread per face (the classifier is two FP64 forward passes per face),
// then one thread per cell for the difference and the RK3 stage.  Every
// operation is an explicit round-to-nearest intrinsic in the oracle's order
// (fp64_ops.cuh), so results are bit-identical to the oracle.
#include "fp64_ops.cuh"
#include "internal.h"

namespace neno6 {
namespace {

using namespace f64ops;

__global__ void __launch_bounds__(128) scalar_faces_kernel(const __grid_constant__ ScalarParams P) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.a.nx;
  if (f > n) return;
  double uu[6], fl[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    uu[k] = P.u[wrap_index(f - 3 + k, n, P.a.bcx)];
    fl[k] = P.law == 0 ? uu[k] : __dmul_rn(0.5, __dmul_rn(uu[k], uu[k]));
  }
  double alpha = 1.0;
  if (P.law != 0) {
    alpha = dabs(uu[0]);
#pragma unroll
    for (int k = 1; k < 6; ++k) alpha = dmax_nn(alpha, dabs(uu[k]));
  }
  double sp[6], sn[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    sp[k] = __dmul_rn(0.5, __fma_rn(alpha, uu[k], fl[k]));
    sn[5 - k] = __dmul_rn(0.5, __fma_rn(-alpha, uu[k], fl[k]));  // mirrored "-" side
  }
  unsigned ep, em;
  if (P.a.mask_mode == kMaskSmooth) {
    ep = em = 0u;
  } else if (P.a.mask_mode == kMaskRough) {
    ep = em = 15u;
  } else if (P.a.mask_mode == kMaskTeno) {
    ep = teno6_eta(P.a.teno, sp);
    em = teno6_eta(P.a.teno, sn);
  } else {
    double x[6], z[4];
    normalise6(sp, x);
    ep = mlp64(P.net.p, x, z);
    normalise6(sn, x);
    em = mlp64(P.net.p, x, z);
  }
  P.F[f] = __dadd_rn(combine64(P.a, sp, ep), combine64(P.a, sn, em));
  if (P.mask_out) P.mask_out[f] = (uint8_t)(ep | (em << 4));
}

// du/dt = -(F_{i+1/2} - F_{i-1/2}) / dx and, for stage > 0, the SSP-RK3
// stage with step h: 1: u1 = u + h L(u); 2: u2 = 3/4 u + 1/4 (u1 + h L(u1));
// 3: u = 1/3 u + 2/3 (u2 + h L(u2)).  `in` is the stage input, `u0` the
// step's start, `out` the result.
__global__ void __launch_bounds__(256) scalar_diff_kernel(const double* __restrict__ F, const double* in,
                                                          const double* u0, double* out, int n, double dx,
                                                          int stage, double h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double L = -__ddiv_rn(__dsub_rn(F[i + 1], F[i]), dx);
  double v = L;
  if (stage == 1) v = __fma_rn(h, L, in[i]);
  else if (stage == 2) v = __fma_rn(0.75, u0[i], __dmul_rn(0.25, __fma_rn(h, L, in[i])));
  else if (stage == 3) v = __fma_rn(1.0 / 3.0, u0[i], __dmul_rn(2.0 / 3.0, __fma_rn(h, L, in[i])));
  out[i] = v;
}

// max over the cells of |f'(u)| as a bit pattern (non-negative binary64
// values order like their patterns).
__global__ void __launch_bounds__(256) scalar_speed_kernel(const double* __restrict__ u, int n, int law,
                                                           unsigned long long* amax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long m = 0ull;
  if (i < n) m = (unsigned long long)dbits(law == 0 ? 1.0 : dabs(u[i]));
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(amax, m);
}

}  // namespace

cudaError_t launch_scalar_faces(const ScalarParams& p, cudaStream_t s) {
  const int faces = p.a.nx + 1;
  scalar_faces_kernel<<<(faces + 127) / 128, 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_scalar_diff(const double* F, const double* in, const double* u0, double* out, int n,
                               double dx, int stage, double h, cudaStream_t s) {
  scalar_diff_kernel<<<(n + 255) / 256, 256, 0, s>>>(F, in, u0, out, n, dx, stage, h);
  return cudaGetLastError();
}

cudaError_t launch_scalar_speed(const double* u, int n, int law, unsigned long long* amax, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  scalar_speed_kernel<<<(n + 255) / 256, 256, 0, s>>>(u, n, law, amax);
  return cudaGetLastError();
}

}  // namespace neno6
