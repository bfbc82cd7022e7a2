// FP64 building blocks shared by the FP64 right-hand-side kernels (fp64.cu)
// and the scalar-law kernels (scalar.cu): the classifier, the normalisation
// of its input and the candidate combination, every operation an explicit
// round-to-nearest intrinsic in the canonical order the oracle follows, so
// both kernel families reproduce the oracle bit for bit.  Translation units
// that include this compile with -fmad=false.
#pragma once

#include "internal.h"

namespace neno6 {
namespace f64ops {

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// x > 0 for every non-NaN x (sign bit clear and not +0).
__device__ __forceinline__ bool gt0(double x) { return dbits(x) > 0; }
__device__ __forceinline__ double relu(double x) { return gt0(x) ? x : 0.0; }
__device__ __forceinline__ double dabs(double x) {
  return __longlong_as_double(dbits(x) & 0x7fffffffffffffffLL);
}
// max of two non-negative values (bit patterns order like the values).
__device__ __forceinline__ double dmax_nn(double a, double b) { return dbits(b) > dbits(a) ? b : a; }

__device__ __forceinline__ int wrap_index(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// beta = v^T B v, summed row by row in index order (an integral of squared
// derivatives: a value that rounds below 0 is 0).
template <int R>
__device__ __forceinline__ double quad_form_rn(const double* __restrict__ B, const double* v) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    double row = 0.0;
#pragma unroll
    for (int j = 0; j < R; ++j) row = __dadd_rn(row, __dmul_rn(B[i * R + j], v[j]));
    s = __dadd_rn(s, __dmul_rn(v[i], row));
  }
  return s > 0.0 ? s : 0.0;
}

// TENO6-opt stencil selection (Sec. 2.1-2.2) on the six values s (i-2..i+3),
// returned as eta bits (bit k set <=> S_k discarded):
//   tau_6 = |beta_6 - (beta_1 + beta_2 + 4 beta_0) / 6|      Eq. (taukTENO)
//   gamma_k = (1 + tau_6 / (beta_k + 1e-40))^6               Eq. (measureTENO)
//   chi_k = gamma_k / sum gamma, delta_k = [chi_k >= 1e-6]   Eqs. (normalize), (cut-off)
// with gamma_k / gamma_max = (a_k / a_max)^6 (three multiplications) in
// the ratio, which cannot overflow.  T: the kTenoTable indicator matrices.
__device__ __forceinline__ unsigned teno6_eta(const double* __restrict__ T, const double s[6]) {
  double beta[4], v[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c0 = k == 0 ? 1 : (k == 1 ? 2 : 0);
#pragma unroll
    for (int j = 0; j < 3; ++j) v[j] = __dsub_rn(s[c0 + j], s[c0]);
    beta[k] = quad_form_rn<3>(T + 9 * k, v);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __dsub_rn(s[2 + j], s[2]);
  beta[3] = quad_form_rn<4>(T + 27, v);
#pragma unroll
  for (int j = 0; j < 6; ++j) v[j] = __dsub_rn(s[j], s[0]);
  const double beta6 = quad_form_rn<6>(T + 43, v);
  double t = __dadd_rn(beta[1], beta[2]);
  t = __dadd_rn(t, __dmul_rn(4.0, beta[0]));
  t = __ddiv_rn(t, 6.0);
  const double tau = dabs(__dsub_rn(beta6, t));
  double a[4], amax = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = __dadd_rn(1.0, __ddiv_rn(tau, __dadd_rn(beta[k], 1e-40)));
    amax = k == 0 ? a[k] : dmax_nn(amax, a[k]);
  }
  double g[4], sum = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double b = __ddiv_rn(a[k], amax);
    const double b2 = __dmul_rn(b, b);
    const double b3 = __dmul_rn(b2, b);
    g[k] = __dmul_rn(b3, b3);
    sum = __dadd_rn(sum, g[k]);
  }
  unsigned eta = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!(__ddiv_rn(g[k], sum) >= 1e-6)) eta |= 1u << k;
  return eta;
}

// Classifier 6-64-32-16-8-4 of Sec. 3.1 on a normalised stencil.  Eq.
// (reconstuction): every output of a layer is its bias followed by an fma
// chain over the layer's inputs in ascending order; ReLU (Eq.
// (activationfunction)) on hidden layers.  Layers 1+2 and 3+4 are fused: each
// hidden unit of layer 1 (3) is completed and immediately accumulated into
// all sums of layer 2 (4), which keeps every sum's term order unchanged while
// holding ~40 values live instead of ~100.  Parameters are packed per layer
// as W[out][in] then b[out]: offsets 0/384, 448/2496, 2528/3040, 3056/3184,
// 3192/3224.  Returns eta bits (logit > 0 <=> sigmoid > 1/2 <=> discard).
__device__ __forceinline__ unsigned mlp64(const double* __restrict__ W, const double* x, double* z) {
  double a2[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) a2[o] = W[2496 + o];
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    double h = W[384 + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) h = __fma_rn(W[i * 6 + k], x[k], h);
    h = relu(h);
#pragma unroll
    for (int o = 0; o < 32; ++o) a2[o] = __fma_rn(W[448 + o * 64 + i], h, a2[o]);
  }
#pragma unroll
  for (int o = 0; o < 32; ++o) a2[o] = relu(a2[o]);
  double a4[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) a4[o] = W[3184 + o];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    double h = W[3040 + j];
#pragma unroll
    for (int i = 0; i < 32; ++i) h = __fma_rn(W[2528 + j * 32 + i], a2[i], h);
    h = relu(h);
#pragma unroll
    for (int o = 0; o < 8; ++o) a4[o] = __fma_rn(W[3056 + o * 16 + j], h, a4[o]);
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) a4[o] = relu(a4[o]);
  unsigned eta = 0;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    double acc = W[3224 + o];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc = __fma_rn(W[3192 + o * 8 + i], a4[i], acc);
    z[o] = acc;
    eta |= (gt0(acc) ? 1u : 0u) << o;
  }
  return eta;
}

// The 6-32-32-32-4 classifier of the width study, same arithmetic order
// (bias, then an fma chain over the inputs in ascending order; ReLU on hidden
// layers); layers 1+2 and 3+4 fused as in mlp64.  Packed offsets: W1 0 /
// b1 192, W2 224 / b2 1248, W3 1280 / b3 2304, W4 2336 / b4 2464.
__device__ __forceinline__ unsigned mlp64_narrow(const double* __restrict__ W, const double* x, double* z) {
  double a2[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) a2[o] = W[1248 + o];
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    double h = W[192 + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) h = __fma_rn(W[i * 6 + k], x[k], h);
    h = relu(h);
#pragma unroll
    for (int o = 0; o < 32; ++o) a2[o] = __fma_rn(W[224 + o * 32 + i], h, a2[o]);
  }
#pragma unroll
  for (int o = 0; o < 32; ++o) a2[o] = relu(a2[o]);
  double a4[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) a4[o] = W[2464 + o];
#pragma unroll 4
  for (int j = 0; j < 32; ++j) {
    double h = W[2304 + j];
#pragma unroll
    for (int i = 0; i < 32; ++i) h = __fma_rn(W[1280 + j * 32 + i], a2[i], h);
    h = relu(h);
#pragma unroll
    for (int o = 0; o < 4; ++o) a4[o] = __fma_rn(W[2336 + o * 32 + j], h, a4[o]);
  }
  unsigned eta = 0;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    z[o] = a4[o];
    eta |= (gt0(a4[o]) ? 1u : 0u) << o;
  }
  return eta;
}

// Eq. (normalizainput): divide by max(|s_0|, ..., |s_5|, 1).  s/1 == s
// exactly, so the division is skipped when the maximum is 1.
__device__ __forceinline__ void normalise6(const double* s, double* x) {
  double m = 1.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) m = dmax_nn(m, dabs(s[j]));
  if (dbits(m) == dbits(1.0)) {
#pragma unroll
    for (int j = 0; j < 6; ++j) x[j] = s[j];
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) x[j] = __ddiv_rn(s[j], m);
  }
}

// Candidate fluxes (Eqs. (definitionEq)/(approximatepolynomial)) on the
// stencil s_0..s_5 = i-2..i+3 and their renormalised convex combination
// (Eqs. (TENOweight_renormalize), (convex)); Algorithm 2's first-order
// fallback when all four are discarded.
__device__ __forceinline__ double combine64(const RhsArgs& a, const double* s, unsigned eta) {
  if (eta == 15u) return s[2];
  double f[4];
  f[0] = __fma_rn(a.cand[0][2], s[3], __fma_rn(a.cand[0][1], s[2], __dmul_rn(a.cand[0][0], s[1])));
  f[1] = __fma_rn(a.cand[1][2], s[4], __fma_rn(a.cand[1][1], s[3], __dmul_rn(a.cand[1][0], s[2])));
  f[2] = __fma_rn(a.cand[2][2], s[2], __fma_rn(a.cand[2][1], s[1], __dmul_rn(a.cand[2][0], s[0])));
  f[3] = __fma_rn(a.cand[3][3], s[5],
                  __fma_rn(a.cand[3][2], s[4],
                           __fma_rn(a.cand[3][1], s[3], __dmul_rn(a.cand[3][0], s[2]))));
  double g = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!((eta >> k) & 1u)) g = __fma_rn(a.wtab[eta][k], f[k], g);
  return g;
}

}  // namespace f64ops
}  // namespace neno6
