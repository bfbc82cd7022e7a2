// Frozen-mask adjoint of the FP64 NENO6 right-hand side: grad_U = J^T lambda,
// J = dL(U)/dU with the classifier bits and the LLF alpha argmax held at
// their values for U (the mask is piecewise constant in U, so this is the
// derivative of the scheme wherever it exists).
//
// dU_i/dt = -(F_{i+1/2} - F_{i-1/2})/dx - (G_{j+1/2} - G_{j-1/2})/dy, so the
// cotangent of face f (between cells f-1 and f) is (lambda_f - lambda_{f-1})/dx
// (lambda of a cell outside the grid taken as 0).  Each face flux depends on
// its six stencil cells; its local Jacobian with respect to one cell is
// evaluated exactly by forward-mode dual numbers carrying nv tangents (one
// per conserved variable of that cell), recomputing the face from the state
// (halo recomputation, nothing stored by the forward pass).
//
// Scatter-free: one thread per output cell gathers, over every face whose
// stencil contains the cell (at most six x faces and six y faces, more on
// tiny periodic grids or at transmissive boundaries where ghost cells alias
// the edge cell), the cotangent-weighted column of that face's Jacobian.
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

// Face flux from six stencil cells with a frozen mask (eta+ | eta- << 4 per
// field); the same operations, in the same order, as the forward FP64 path.
template <int NV, int K>
__device__ void face_flux_dual(const CellT<NV, K> (&st)[6], int dir, const RhsArgs& a,
                               const unsigned (&eta)[NV], Dual<K> (&Fh)[NV]) {
  const CellT<NV, K>& A = st[2];
  const CellT<NV, K>& B = st[3];
  const Dual<K> gm1 = dconst<K>(a.gm1);
  Dual<K> den = A.s + B.s;
  Dual<K> ut = dfma(B.s, B.u, A.s * A.u) / den;
  Dual<K> Ht = dfma(B.s, B.H, A.s * A.H) / den;
  Dual<K> vt = dconst<K>(0.0), qt;
  if (NV == 4) {
    vt = dfma(B.s, B.v, A.s * A.v) / den;
    qt = dfma(vt, vt, ut * ut);
  } else {
    qt = ut * ut;
  }
  Dual<K> c2 = gm1 * (Ht - scale(0.5, qt));
  Dual<K> ct = dsqrt(c2);
  Dual<K> ic = dconst<K>(1.0) / ct;
  Dual<K> b1 = gm1 / c2;
  Dual<K> b2 = scale(0.5, b1 * qt);
  Dual<K> nt = (NV == 4 && dir == 1) ? vt : ut;
  Dual<K> nc = nt * ic;
  Dual<K> b1u = b1 * ut, b1v = b1 * vt;
  Dual<K> hb1 = scale(0.5, b1), ntc = nt * ct;
  Dual<K> L[4][4], R[4][4];
  const Dual<K> zero = dconst<K>(0.0), one = dconst<K>(1.0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) L[i][j] = R[i][j] = zero;
  if (NV == 3) {
    L[0][0] = scale(0.5, b2 + nc); L[0][1] = scale(0.5, -b1u - ic); L[0][2] = hb1;
    L[1][0] = one - b2; L[1][1] = b1u; L[1][2] = -b1;
    L[2][0] = scale(0.5, b2 - nc); L[2][1] = scale(0.5, -b1u + ic); L[2][2] = hb1;
    R[0][0] = one; R[0][1] = one; R[0][2] = one;
    R[1][0] = ut - ct; R[1][1] = ut; R[1][2] = ut + ct;
    R[2][0] = Ht - ntc; R[2][1] = scale(0.5, qt); R[2][2] = Ht + ntc;
  } else if (dir == 0) {
    L[0][0] = scale(0.5, b2 + nc); L[0][1] = scale(0.5, -b1u - ic); L[0][2] = scale(0.5, -b1v); L[0][3] = hb1;
    L[1][0] = one - b2; L[1][1] = b1u; L[1][2] = b1v; L[1][3] = -b1;
    L[2][0] = -vt; L[2][1] = zero; L[2][2] = one; L[2][3] = zero;
    L[3][0] = scale(0.5, b2 - nc); L[3][1] = scale(0.5, -b1u + ic); L[3][2] = scale(0.5, -b1v); L[3][3] = hb1;
    R[0][0] = one; R[0][1] = one; R[0][2] = zero; R[0][3] = one;
    R[1][0] = ut - ct; R[1][1] = ut; R[1][2] = zero; R[1][3] = ut + ct;
    R[2][0] = vt; R[2][1] = vt; R[2][2] = one; R[2][3] = vt;
    R[3][0] = Ht - ntc; R[3][1] = scale(0.5, qt); R[3][2] = vt; R[3][3] = Ht + ntc;
  } else {
    L[0][0] = scale(0.5, b2 + nc); L[0][1] = scale(0.5, -b1u); L[0][2] = scale(0.5, -b1v - ic); L[0][3] = hb1;
    L[1][0] = one - b2; L[1][1] = b1u; L[1][2] = b1v; L[1][3] = -b1;
    L[2][0] = -ut; L[2][1] = one; L[2][2] = zero; L[2][3] = zero;
    L[3][0] = scale(0.5, b2 - nc); L[3][1] = scale(0.5, -b1u); L[3][2] = scale(0.5, -b1v + ic); L[3][3] = hb1;
    R[0][0] = one; R[0][1] = one; R[0][2] = zero; R[0][3] = one;
    R[1][0] = ut; R[1][1] = ut; R[1][2] = one; R[1][3] = ut;
    R[2][0] = vt - ct; R[2][1] = vt; R[2][2] = zero; R[2][3] = vt + ct;
    R[3][0] = Ht - ntc; R[3][1] = scale(0.5, qt); R[3][2] = ut; R[3][3] = Ht + ntc;
  }
  Dual<K> gh[NV];
#pragma unroll 1
  for (int m = 0; m < NV; ++m) {
    // alpha_m = max_j |lambda_m(U_j)|, first index wins ties (argmax frozen)
    Dual<K> alpha;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      Dual<K> lam = m == 0 ? st[j].un - st[j].c : (m == NV - 1 ? st[j].un + st[j].c : st[j].un);
      lam = dabs(lam);
      if (j == 0 || lam.v > alpha.v) alpha = lam;
    }
    Dual<K> sp[6], sm[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      Dual<K> vv = L[m][0] * st[j].U[0];
      Dual<K> gg = L[m][0] * st[j].F[0];
#pragma unroll
      for (int n = 1; n < NV; ++n) {
        vv = dfma(L[m][n], st[j].U[n], vv);
        gg = dfma(L[m][n], st[j].F[n], gg);
      }
      sp[j] = scale(0.5, dfma(alpha, vv, gg));
      sm[j] = scale(0.5, dfma(-alpha, vv, gg));
    }
    Dual<K> g2[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      Dual<K> s[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) s[j] = side ? sm[5 - j] : sp[j];
      const unsigned e = side ? (eta[m] >> 4) : (eta[m] & 15u);
      if (e == 15u) {
        g2[side] = s[2];
      } else {
        Dual<K> f[4];
        f[0] = dfma(dconst<K>(a.cand[0][2]), s[3], dfma(dconst<K>(a.cand[0][1]), s[2], dconst<K>(a.cand[0][0]) * s[1]));
        f[1] = dfma(dconst<K>(a.cand[1][2]), s[4], dfma(dconst<K>(a.cand[1][1]), s[3], dconst<K>(a.cand[1][0]) * s[2]));
        f[2] = dfma(dconst<K>(a.cand[2][2]), s[2], dfma(dconst<K>(a.cand[2][1]), s[1], dconst<K>(a.cand[2][0]) * s[0]));
        f[3] = dfma(dconst<K>(a.cand[3][3]), s[5],
                    dfma(dconst<K>(a.cand[3][2]), s[4],
                         dfma(dconst<K>(a.cand[3][1]), s[3], dconst<K>(a.cand[3][0]) * s[2])));
        Dual<K> g = zero;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (!((e >> k) & 1u)) g = dfma(dconst<K>(a.wtab[e][k]), f[k], g);
        g2[side] = g;
      }
    }
    gh[m] = g2[0] + g2[1];
  }
#pragma unroll
  for (int n = 0; n < NV; ++n) {
    Dual<K> acc = R[n][0] * gh[0];
#pragma unroll
    for (int m = 1; m < NV; ++m) acc = dfma(R[n][m], gh[m], acc);
    Fh[n] = acc;
  }
}

// One output cell: gather J^T lambda over the faces of both directions.
template <int NDIM>
__global__ void __launch_bounds__(128) rhs_vjp_kernel(const __grid_constant__ RhsArgs a, const double* __restrict__ lam,
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
#pragma unroll 1
  for (int dir = 0; dir < NDIM; ++dir) {
    const int N = dir == 0 ? nx : ny;     // cells along the sweep line
    const int bc = dir == 0 ? a.bcx : a.bcy;
    const int me = dir == 0 ? ci : cj;    // this cell's index along the line
    const int line = dir == 0 ? cj : ci;  // the line's index across
    const double invd = dir == 0 ? 1.0 / a.dx : 1.0 / a.dy;
    // candidate faces: the direct window, and its periodic images
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
        // stencil slots of face f that alias this cell
        unsigned slots = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (wrapi(f - 3 + k, N, bc) == me) slots |= 1u << k;
        if (!slots) continue;
        // face cotangent (lambda_f - lambda_{f-1}) / d, zero outside the grid
        double Fbar[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
          double lr = 0.0, ll = 0.0;
          if (f < N) lr = dir == 0 ? lam[n * plane + (size_t)line * nx + f] : lam[n * plane + (size_t)f * nx + line];
          if (f > 0)
            ll = dir == 0 ? lam[n * plane + (size_t)line * nx + f - 1] : lam[n * plane + (size_t)(f - 1) * nx + line];
          Fbar[n] = (lr - ll) * invd;
        }
        // frozen mask of this face
        unsigned eta[NV];
#pragma unroll
        for (int m = 0; m < NV; ++m) {
          size_t idx;
          if (dir == 0) idx = ((size_t)m * ny + line) * (nx + 1) + f;
          else idx = (size_t)NV * ny * (nx + 1) + ((size_t)m * (ny + 1) + f) * nx + line;
          eta[m] = a.mask_in[idx];
        }
        // the six stencil cells, with tangents seeded on every slot that is
        // this cell
        CellT<NV, NV> st[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int g = wrapi(f - 3 + k, N, bc);
          const size_t gi = dir == 0 ? (size_t)line * nx + g : (size_t)g * nx + line;
          Dual<NV> U[NV];
#pragma unroll
          for (int n = 0; n < NV; ++n) {
            U[n] = dconst<NV>(a.U[n * plane + gi]);
            if ((slots >> k) & 1u) U[n].d[n] = 1.0;
          }
          cell_state<NV, NV>(U, dir, a.gamma, a.gm1, st[k]);
        }
        Dual<NV> Fh[NV];
        face_flux_dual<NV, NV>(st, dir, a, eta, Fh);
#pragma unroll
        for (int o = 0; o < NV; ++o)
#pragma unroll
          for (int n = 0; n < NV; ++n) acc[n] += Fbar[o] * Fh[o].d[n];
      }
    }
  }
#pragma unroll
  for (int n = 0; n < NV; ++n) grad[n * plane + cell] = acc[n];
}

}  // namespace

cudaError_t launch_rhs_vjp(int ndim, const RhsArgs& a, const double* lam, double* grad, cudaStream_t s) {
  const size_t cells = (size_t)a.nx * a.ny;
  const unsigned blocks = (unsigned)((cells + 127) / 128);
  if (ndim == 2) rhs_vjp_kernel<2><<<blocks, 128, 0, s>>>(a, lam, grad);
  else rhs_vjp_kernel<1><<<blocks, 128, 0, s>>>(a, lam, grad);
  return cudaGetLastError();
}

}  // namespace neno6
