// Frozen-mask adjoint of the FP64 NENO6 right-hand side: grad_U = J^T lambda,
// J = dL(U)/dU with the classifier bits and the LLF alpha argmax held at
// their values for U (the mask is piecewise constant in U, so this is the
// derivative of the scheme wherever it exists).
//
// dU_i/dt = -(F_{i+1/2} - F_{i-1/2})/dx - (G_{j+1/2} - G_{j-1/2})/dy, so the
// cotangent of face f (between cells f-1 and f) is (lambda_f - lambda_{f-1})/d
// (lambda of a cell outside the grid taken as 0).  Each face flux depends on
// its six stencil cells.  Two kernels:
//  * vjp_face_kernel, one thread per face: recomputes the face from U (halo
//    recomputation; the forward pass stores nothing) and runs reverse mode
//    through it, using that with the mask frozen the reconstruction of each
//    side is linear in the six split fluxes; the small nonlinear pieces (a
//    cell's state and flux, the Roe average) are differentiated by
//    forward-mode dual numbers with one tangent per conserved variable.  It
//    writes the face's contribution to each of its six cells;
//  * vjp_gather_kernel, one thread per cell: adds the contributions of every
//    face whose stencil holds the cell (six per direction, more where
//    periodic images or zero-gradient ghost cells alias it) in a fixed order.
// Every output is written once; there are no atomics and the result is
// deterministic.
#include "internal.h"

namespace neno6 {
namespace {

template <int K>
struct Dual {
  double v;
  double d[K];
};

template <int K>
__device__ __forceinline__ Dual<K> dconst(double x) {
  Dual<K> r;
  r.v = x;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = 0.0;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = __dadd_rn(a.v, b.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = __dsub_rn(a.v, b.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = __dmul_rn(a.v, b.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = __ddiv_rn(a.v, b.v);
  const double inv = 1.0 / b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> dfma(const Dual<K>& a, const Dual<K>& b, const Dual<K>& c) {
  Dual<K> r;
  r.v = __fma_rn(a.v, b.v, c.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k] + c.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> dsqrt(const Dual<K>& a) {
  Dual<K> r;
  r.v = __dsqrt_rn(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> dabs(const Dual<K>& a) {
  return a.v < 0.0 ? -a : a;
}
template <int K>
__device__ __forceinline__ Dual<K> scale(double s, const Dual<K>& a) {  // exact constant factor
  Dual<K> r;
  r.v = __dmul_rn(s, a.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = s * a.d[k];
  return r;
}

__device__ __forceinline__ int wrapi(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Per-cell state (Sec. 4.4): velocities, sound speed, enthalpy, sqrt(rho),
// physical flux in direction dir.
template <int NV, int K>
struct CellT {
  Dual<K> U[NV], F[NV], un, u, v, c, H, s;
};

template <int NV, int K>
__device__ __forceinline__ void cell_state(const Dual<K> (&U)[NV], int dir, double gamma, double gm1,
                                           CellT<NV, K>& o) {
#pragma unroll
  for (int n = 0; n < NV; ++n) o.U[n] = U[n];
  const Dual<K>& rho = U[0];
  const Dual<K>& E = U[NV - 1];
  Dual<K> u = U[1] / rho;
  Dual<K> v = dconst<K>(0.0), q;
  if (NV == 4) {
    v = U[2] / rho;
    q = dfma(v, v, u * u);
  } else {
    q = u * u;
  }
  Dual<K> p = dconst<K>(gm1) * (E - dconst<K>(0.5) * (rho * q));
  o.c = dsqrt((dconst<K>(gamma) * p) / rho);
  Dual<K> Ep = E + p;
  o.u = u;
  o.v = v;
  o.H = Ep / rho;
  o.s = dsqrt(rho);
  if (NV == 3) {
    o.un = u;
    o.F[0] = U[1];
    o.F[1] = dfma(U[1], u, p);
    o.F[2] = Ep * u;
  } else if (dir == 0) {
    o.un = u;
    o.F[0] = U[1];
    o.F[1] = dfma(U[1], u, p);
    o.F[2] = U[2] * u;
    o.F[NV - 1] = Ep * u;
  } else {
    o.un = v;
    o.F[0] = U[2];
    o.F[1] = U[1] * v;
    o.F[2] = dfma(U[2], v, p);
    o.F[NV - 1] = Ep * v;
  }
}

// Roe-averaged quantities of the face between cells A (left) and B (right),
// in the forward FP64 path's order (Sec. 4.4; eigenvectors in the Roe/Toro
// form, b1 = (gamma-1)/c^2, b2 = b1 |u|^2 / 2).
template <int K>
struct RoeT {
  Dual<K> ut, vt, Ht, qt, ct, ic, b1, b2, nc, b1u, b1v, hb1, ntc;
};

template <int NV, int K>
__device__ __forceinline__ void roe_avg(const CellT<NV, K>& A, const CellT<NV, K>& B, int dir, double gm1_,
                                        RoeT<K>& r) {
  const Dual<K> gm1 = dconst<K>(gm1_);
  const Dual<K> den = A.s + B.s;
  r.ut = dfma(B.s, B.u, A.s * A.u) / den;
  r.Ht = dfma(B.s, B.H, A.s * A.H) / den;
  r.vt = dconst<K>(0.0);
  if (NV == 4) {
    r.vt = dfma(B.s, B.v, A.s * A.v) / den;
    r.qt = dfma(r.vt, r.vt, r.ut * r.ut);
  } else {
    r.qt = r.ut * r.ut;
  }
  const Dual<K> c2 = gm1 * (r.Ht - scale(0.5, r.qt));
  r.ct = dsqrt(c2);
  r.ic = dconst<K>(1.0) / r.ct;
  r.b1 = gm1 / c2;
  r.b2 = scale(0.5, r.b1 * r.qt);
  const Dual<K> nt = (NV == 4 && dir == 1) ? r.vt : r.ut;
  r.nc = nt * r.ic;
  r.b1u = r.b1 * r.ut;
  r.b1v = r.b1 * r.vt;
  r.hb1 = scale(0.5, r.b1);
  r.ntc = nt * r.ct;
}

// Row m of L = R^-1 (characteristic field m: u_n - c, entropy, [shear,] u_n + c).
template <int NV, int K>
__device__ __forceinline__ void L_row(const RoeT<K>& r, int dir, int m, Dual<K> (&row)[4]) {
  const Dual<K> zero = dconst<K>(0.0), one = dconst<K>(1.0);
  row[3] = zero;
  if (NV == 3) {
    if (m == 0) { row[0] = scale(0.5, r.b2 + r.nc); row[1] = scale(0.5, -r.b1u - r.ic); row[2] = r.hb1; }
    else if (m == 1) { row[0] = one - r.b2; row[1] = r.b1u; row[2] = -r.b1; }
    else { row[0] = scale(0.5, r.b2 - r.nc); row[1] = scale(0.5, -r.b1u + r.ic); row[2] = r.hb1; }
  } else if (dir == 0) {
    if (m == 0) { row[0] = scale(0.5, r.b2 + r.nc); row[1] = scale(0.5, -r.b1u - r.ic); row[2] = scale(0.5, -r.b1v); row[3] = r.hb1; }
    else if (m == 1) { row[0] = one - r.b2; row[1] = r.b1u; row[2] = r.b1v; row[3] = -r.b1; }
    else if (m == 2) { row[0] = -r.vt; row[1] = zero; row[2] = one; }
    else { row[0] = scale(0.5, r.b2 - r.nc); row[1] = scale(0.5, -r.b1u + r.ic); row[2] = scale(0.5, -r.b1v); row[3] = r.hb1; }
  } else {
    if (m == 0) { row[0] = scale(0.5, r.b2 + r.nc); row[1] = scale(0.5, -r.b1u); row[2] = scale(0.5, -r.b1v - r.ic); row[3] = r.hb1; }
    else if (m == 1) { row[0] = one - r.b2; row[1] = r.b1u; row[2] = r.b1v; row[3] = -r.b1; }
    else if (m == 2) { row[0] = -r.ut; row[1] = one; row[2] = zero; }
    else { row[0] = scale(0.5, r.b2 - r.nc); row[1] = scale(0.5, -r.b1u); row[2] = scale(0.5, -r.b1v + r.ic); row[3] = r.hb1; }
  }
}

// Column m of R (right eigenvectors).
template <int NV, int K>
__device__ __forceinline__ void R_col(const RoeT<K>& r, int dir, int m, Dual<K> (&col)[4]) {
  const Dual<K> zero = dconst<K>(0.0), one = dconst<K>(1.0);
  col[3] = zero;
  if (NV == 3) {
    if (m == 0) { col[0] = one; col[1] = r.ut - r.ct; col[2] = r.Ht - r.ntc; }
    else if (m == 1) { col[0] = one; col[1] = r.ut; col[2] = scale(0.5, r.qt); }
    else { col[0] = one; col[1] = r.ut + r.ct; col[2] = r.Ht + r.ntc; }
  } else if (dir == 0) {
    if (m == 0) { col[0] = one; col[1] = r.ut - r.ct; col[2] = r.vt; col[3] = r.Ht - r.ntc; }
    else if (m == 1) { col[0] = one; col[1] = r.ut; col[2] = r.vt; col[3] = scale(0.5, r.qt); }
    else if (m == 2) { col[0] = zero; col[1] = zero; col[2] = one; col[3] = r.vt; }
    else { col[0] = one; col[1] = r.ut + r.ct; col[2] = r.vt; col[3] = r.Ht + r.ntc; }
  } else {
    if (m == 0) { col[0] = one; col[1] = r.ut; col[2] = r.vt - r.ct; col[3] = r.Ht - r.ntc; }
    else if (m == 1) { col[0] = one; col[1] = r.ut; col[2] = r.vt; col[3] = scale(0.5, r.qt); }
    else if (m == 2) { col[0] = zero; col[1] = one; col[2] = zero; col[3] = r.ut; }
    else { col[0] = one; col[1] = r.ut; col[2] = r.vt + r.ct; col[3] = r.Ht + r.ntc; }
  }
}

// With the mask frozen, one side's reconstruction is linear in its six split
// fluxes: g_hat = sum_j c_j s_j, c_j = sum over kept stencils k of
// w_k(eta) times S_k's candidate coefficient on point j (Eqs. (convex),
// (TENOweight_renormalize)); all stencils discarded: c = e_2 (first-order
// fallback, Algorithm 2).
__device__ __forceinline__ void side_coeffs(unsigned e, const RhsArgs& a, double (&c)[6]) {
#pragma unroll
  for (int j = 0; j < 6; ++j) c[j] = 0.0;
  if (e == 15u) {
    c[2] = 1.0;
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if ((e >> k) & 1u) continue;
    // S_0 = {i-1, i, i+1}, S_1 = {i, i+1, i+2}, S_2 = {i-2, i-1, i},
    // S_3 = {i, ..., i+3}; stencil point j = 0..5 is cell i-2+j
    const int start = k == 0 ? 1 : (k == 2 ? 0 : 2);
    const int len = k == 3 ? 4 : 3;
    const double w = a.wtab[e][k];
#pragma unroll
    for (int l = 0; l < 4; ++l)
      if (l < len) c[start + l] = __fma_rn(w, a.cand[k][l], c[start + l]);
  }
}

constexpr int kVjpThreads = 128;

// Reverse mode over one face (one thread per face): the face's share of
// J^T lambda for each of its six stencil cells, written to
// contrib[(slot * nv + n) * nfaces + face].  With the mask frozen the face
// flux is
//   F_hat = sum_m R_m g_m,  g_m = (L_m . P_m + alpha_m L_m . Q_m) / 2,
//   P_m = sum_j (c+_j + c-_j) F_j,  Q_m = sum_j (c+_j - c-_j) U_j,
// (c+ the "+" side's coefficients on points i-2..i+3, c- the "-" side's
// mirrored), alpha_m = |lambda_m| of the stencil cell holding the maximum.
// Given the face cotangent Fbar = (lambda_f - lambda_{f-1})/d:
//   gbar_m = R_m . Fbar;  Pbar_m = gbar_m L_m / 2;  Qbar_m = alpha_m Pbar_m;
//   alphabar_m = gbar_m (L_m . Q_m) / 2;
// the cells receive Pbar through their flux Jacobians (forward-mode duals of
// the cell state), Qbar directly, alphabar through d|lambda_m|/dU of the
// argmax cell, and cells i, i+1 the derivative of the Roe average through
// Phi = sum_m (Fbar . R_m) (L_m . (P_m + alpha_m Q_m)) / 2 with P, Q, alpha
// held fixed (forward-mode duals seeded on the cell).
template <int NDIM>
__global__ void __launch_bounds__(kVjpThreads) vjp_face_kernel(const __grid_constant__ RhsArgs a,
                                                               const double* __restrict__ lam,
                                                               double* __restrict__ contrib, int dir) {
  constexpr int NV = NDIM == 2 ? 4 : 3;
  extern __shared__ double vsm[];
  const int t = threadIdx.x;
  // per-thread columns: U_j[n], F_j[n], Ubar_j[n] at row (j * NV + n)
  auto sU = [&](int j, int n) -> double& { return vsm[(j * NV + n) * kVjpThreads + t]; };
  auto sF = [&](int j, int n) -> double& { return vsm[((6 + j) * NV + n) * kVjpThreads + t]; };
  auto sB = [&](int j, int n) -> double& { return vsm[((12 + j) * NV + n) * kVjpThreads + t]; };
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const int N = dir == 0 ? nx : ny;      // cells along a line
  const int nl = dir == 0 ? ny : nx;     // lines
  const int bc = dir == 0 ? a.bcx : a.bcy;
  const long long nfaces = (long long)(N + 1) * nl;
  const long long id = (long long)blockIdx.x * kVjpThreads + t;
  if (id >= nfaces) return;
  // x faces: id = line * (nx + 1) + f;  y faces: id = f * nx + line
  const int f = dir == 0 ? (int)(id % (N + 1)) : (int)(id / nl);
  const int line = dir == 0 ? (int)(id / (N + 1)) : (int)(id % nl);
  auto cell = [&](int i) -> size_t { return dir == 0 ? (size_t)line * nx + i : (size_t)i * nx + line; };
  const double invd = dir == 0 ? 1.0 / a.dx : 1.0 / a.dy;
  double Fbar[NV];
#pragma unroll
  for (int n = 0; n < NV; ++n) {
    const double lr = f < N ? lam[n * plane + cell(f)] : 0.0;
    const double ll = f > 0 ? lam[n * plane + cell(f - 1)] : 0.0;
    Fbar[n] = (lr - ll) * invd;
  }
  unsigned eta[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    const size_t idx = dir == 0 ? ((size_t)m * ny + line) * (nx + 1) + f
                                : (size_t)NV * ny * (nx + 1) + ((size_t)m * (ny + 1) + f) * nx + line;
    eta[m] = a.mask_in[idx];
  }
  // stencil cells: conserved variables, fluxes and signal speeds (plain)
  double un[6], cs[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const size_t g = cell(wrapi(f - 3 + j, N, bc));
    Dual<1> U[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      U[n] = dconst<1>(a.U[n * plane + g]);
      sU(j, n) = U[n].v;
      sB(j, n) = 0.0;
    }
    CellT<NV, 1> c;
    cell_state<NV, 1>(U, dir, a.gamma, a.gm1, c);
#pragma unroll
    for (int n = 0; n < NV; ++n) sF(j, n) = c.F[n].v;
    un[j] = c.un.v;
    cs[j] = c.c.v;
  }
  // Roe average (plain)
  RoeT<1> r;
  {
    Dual<1> UA[NV], UB[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      UA[n] = dconst<1>(sU(2, n));
      UB[n] = dconst<1>(sU(3, n));
    }
    CellT<NV, 1> A, B;
    cell_state<NV, 1>(UA, dir, a.gamma, a.gm1, A);
    cell_state<NV, 1>(UB, dir, a.gamma, a.gm1, B);
    roe_avg<NV, 1>(A, B, dir, a.gm1, r);
  }
  // pass 1 over the fields: alpha_m and its cell, P_m, Q_m, gbar_m
  double W[NV][NV];  // P_m + alpha_m Q_m
  double abar[NV], gbar[NV], alph[NV];
  int jstar[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    double cp[6], cm[6];
    side_coeffs(eta[m] & 15u, a, cp);
    side_coeffs(eta[m] >> 4, a, cm);
    // alpha_m: the first index of the maximum |lambda_m| wins
    double alpha = 0.0;
    int js = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double l = fabs(m == 0 ? un[j] - cs[j] : (m == NV - 1 ? un[j] + cs[j] : un[j]));
      if (j == 0 || l > alpha) {
        alpha = l;
        js = j;
      }
    }
    jstar[m] = js;
    alph[m] = alpha;
    double P[NV], Q[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      P[n] = 0.0;
      Q[n] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      // the "-" side's point k is stencil point 5 - k
      const double ap = cp[j] + cm[5 - j], am = cp[j] - cm[5 - j];
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        P[n] = __fma_rn(ap, sF(j, n), P[n]);
        Q[n] = __fma_rn(am, sU(j, n), Q[n]);
      }
    }
    Dual<1> Lr[4], Rc[4];
    L_row<NV, 1>(r, dir, m, Lr);
    R_col<NV, 1>(r, dir, m, Rc);
    double LQ = 0.0, gb = 0.0;
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      LQ = __fma_rn(Lr[n].v, Q[n], LQ);
      gb = __fma_rn(Rc[n].v, Fbar[n], gb);
      W[m][n] = __fma_rn(alpha, Q[n], P[n]);
    }
    gbar[m] = gb;
    abar[m] = 0.5 * gb * LQ;
  }
  // pass 2: Pbar_m = gbar_m L_m / 2 to the cells' flux adjoints (sF is free
  // now and holds them), Qbar_m = alpha_m Pbar_m to their U adjoints
#pragma unroll
  for (int j = 0; j < 6; ++j)
#pragma unroll
    for (int n = 0; n < NV; ++n) sF(j, n) = 0.0;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    double cp[6], cm[6];
    side_coeffs(eta[m] & 15u, a, cp);
    side_coeffs(eta[m] >> 4, a, cm);
    Dual<1> Lr[4];
    L_row<NV, 1>(r, dir, m, Lr);
    double pb[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) pb[n] = 0.5 * gbar[m] * Lr[n].v;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double ap = cp[j] + cm[5 - j], am = alph[m] * (cp[j] - cm[5 - j]);
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        sF(j, n) = __fma_rn(ap, pb[n], sF(j, n));
        sB(j, n) = __fma_rn(am, pb[n], sB(j, n));
      }
    }
  }
  // each cell: flux Jacobian^T times its flux adjoint, plus the alpha terms
  // of the fields whose maximum it holds (d|lambda| = sign(lambda) dlambda)
#pragma unroll 1
  for (int j = 0; j < 6; ++j) {
    Dual<NV> U[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      U[n] = dconst<NV>(sU(j, n));
      U[n].d[n] = 1.0;
    }
    CellT<NV, NV> c;
    cell_state<NV, NV>(U, dir, a.gamma, a.gm1, c);
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = sB(j, k);
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      const double fb = sF(j, n);
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = __fma_rn(fb, c.F[n].d[k], acc[k]);
    }
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      if (jstar[m] != j) continue;
      const Dual<NV> l = m == 0 ? c.un - c.c : (m == NV - 1 ? c.un + c.c : c.un);
      const double w = l.v < 0.0 ? -abar[m] : abar[m];
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = __fma_rn(w, l.d[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) sB(j, k) = acc[k];
  }
  // the Roe average: d Phi / dU for cells i (slot 2) and i+1 (slot 3)
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    Dual<NV> UA[NV], UB[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) {
      UA[n] = dconst<NV>(sU(2, n));
      UB[n] = dconst<NV>(sU(3, n));
      if (side == 0) UA[n].d[n] = 1.0;
      else UB[n].d[n] = 1.0;
    }
    RoeT<NV> rr;
    {
      CellT<NV, NV> A, B;
      cell_state<NV, NV>(UA, dir, a.gamma, a.gm1, A);
      cell_state<NV, NV>(UB, dir, a.gamma, a.gm1, B);
      roe_avg<NV, NV>(A, B, dir, a.gm1, rr);
    }
    Dual<NV> phi = dconst<NV>(0.0);
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      Dual<NV> Lr[4], Rc[4];
      L_row<NV, NV>(rr, dir, m, Lr);
      R_col<NV, NV>(rr, dir, m, Rc);
      Dual<NV> y = dconst<NV>(0.0), z = dconst<NV>(0.0);
#pragma unroll
      for (int n = 0; n < NV; ++n) {
        y = dfma(Lr[n], dconst<NV>(W[m][n]), y);
        z = dfma(Rc[n], dconst<NV>(Fbar[n]), z);
      }
      phi = dfma(scale(0.5, z), y, phi);
    }
    const int j = 2 + side;
#pragma unroll
    for (int k = 0; k < NV; ++k) sB(j, k) += phi.d[k];
  }
#pragma unroll
  for (int j = 0; j < 6; ++j)
#pragma unroll
    for (int n = 0; n < NV; ++n) contrib[(size_t)(j * NV + n) * nfaces + id] = sB(j, n);
}

// One output cell: sum, in a fixed order, the contributions of every face
// whose stencil holds the cell (six per direction; more where periodic
// images or zero-gradient ghost cells alias it).  No atomics: deterministic.
template <int NDIM>
__global__ void __launch_bounds__(256) vjp_gather_kernel(const __grid_constant__ RhsArgs a,
                                                         const double* __restrict__ contrib,
                                                         double* __restrict__ grad) {
  constexpr int NV = NDIM == 2 ? 4 : 3;
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= plane) return;
  const int ci = (int)(cell % nx), cj = (int)(cell / nx);
  double acc[NV];
#pragma unroll
  for (int n = 0; n < NV; ++n) acc[n] = 0.0;
  const double* base = contrib;
#pragma unroll 1
  for (int dir = 0; dir < NDIM; ++dir) {
    const int N = dir == 0 ? nx : ny;
    const int nl = dir == 0 ? ny : nx;
    const int bc = dir == 0 ? a.bcx : a.bcy;
    const int me = dir == 0 ? ci : cj;
    const int line = dir == 0 ? cj : ci;
    const long long nfaces = (long long)(N + 1) * nl;
    int lo[3], hi[3], nwin = 0;
    if (N <= 16) {
      lo[0] = 0; hi[0] = N; nwin = 1;
    } else {
      lo[nwin] = max(me - 2, 0); hi[nwin] = min(me + 3, N); ++nwin;
      if (bc == 0) {
        if (me + 3 - N >= 0) { lo[nwin] = 0; hi[nwin] = me + 3 - N; ++nwin; }
        if (me - 2 + N <= N) { lo[nwin] = max(me - 2 + N, 0); hi[nwin] = N; ++nwin; }
      }
      // zero-gradient ghost cells alias the edge cells only from faces
      // 0..3 and N-3..N, which the direct window of an edge cell covers
    }
#pragma unroll 1
    for (int w = 0; w < nwin; ++w) {
#pragma unroll 1
      for (int f = lo[w]; f <= hi[w]; ++f) {
        const long long id = dir == 0 ? (long long)line * (N + 1) + f : (long long)f * nl + line;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          if (wrapi(f - 3 + k, N, bc) != me) continue;
#pragma unroll
          for (int n = 0; n < NV; ++n) acc[n] += base[(size_t)(k * NV + n) * nfaces + id];
        }
      }
    }
    base += (size_t)6 * NV * nfaces;
  }
#pragma unroll
  for (int n = 0; n < NV; ++n) grad[n * plane + cell] = acc[n];
}

}  // namespace

size_t vjp_scratch_bytes(int ndim, int nx, int ny) {
  const int nv = ndim == 2 ? 4 : 3;
  size_t faces = (size_t)(nx + 1) * ny;
  if (ndim == 2) faces += (size_t)(ny + 1) * nx;
  return faces * 6 * nv * sizeof(double);
}

cudaError_t launch_rhs_vjp(int ndim, const RhsArgs& a, const double* lam, double* grad, double* scratch,
                           cudaStream_t s) {
  const int nv = ndim == 2 ? 4 : 3;
  const size_t smem = (size_t)18 * nv * kVjpThreads * sizeof(double);
  auto face = ndim == 2 ? vjp_face_kernel<2> : vjp_face_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(face, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  double* cy = scratch;
  for (int dir = 0; dir < ndim; ++dir) {
    const long long nfaces = dir == 0 ? (long long)(a.nx + 1) * a.ny : (long long)(a.ny + 1) * a.nx;
    const unsigned blocks = (unsigned)((nfaces + kVjpThreads - 1) / kVjpThreads);
    face<<<blocks, kVjpThreads, smem, s>>>(a, lam, cy, dir);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cy += (size_t)6 * nv * nfaces;
  }
  const size_t cells = (size_t)a.nx * a.ny;
  const unsigned gblocks = (unsigned)((cells + 255) / 256);
  if (ndim == 2) vjp_gather_kernel<2><<<gblocks, 256, 0, s>>>(a, scratch, grad);
  else vjp_gather_kernel<1><<<gblocks, 256, 0, s>>>(a, scratch, grad);
  return cudaGetLastError();
}

}  // namespace neno6
