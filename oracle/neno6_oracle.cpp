// NENO6 oracle: a plain, slow FP64 CPU implementation of the NENO6 scheme of
// Li, Fu & Adams, "A six-point neuron-based ENO (NENO6) scheme for compressible
// fluid dynamics" (arXiv 2207.08500).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load this file's library.  The product
// library never links, loads or calls it, and it shares no code with the CUDA
// path: the two are written independently from the same reading of the paper.
//
// What it computes, in the paper's order:
//   * Sec. 2, Eqs. (ordinaryEq)-(approximateEq): the conservative finite
//     difference du_i/dt = -(F_{i+1/2} - F_{i-1/2}) / dx.
//   * Sec. 2, Eq. (convex) with the renormalised weights of
//     Eq. (TENOweight_renormalize): F_{i+1/2} = sum_k w_k F_{k,i+1/2},
//     w_k = d_k delta_k / sum_k d_k delta_k (d_k from Sec. 2.2 / Sec. 4).
//     The candidate-stencil coefficients come in from the caller; they are
//     derived exactly from Eqs. (definitionEq)/(approximatepolynomial) in
//     oracle/coefficients.py.
//   * Sec. 3.1, Eq. (normalizainput): MLP input = the six stencil values
//     divided by max(|f_{i-2}|, ..., |f_{i+3}|, 1).
//   * Sec. 3.1, Eqs. (reconstuction), (activationfunction), (sigmoidfunction):
//     affine layers, ReLU on the hidden layers, sigmoid on the output layer;
//     a stencil is discarded when its probability exceeds 1/2, i.e. when its
//     logit is > 0 (sigmoid is monotone, so exp is never evaluated).
//   * Algorithm 2: features -> prediction -> renormalised convex combination
//     -> first-order upwind flux when all four stencils are discarded.
//   * Sec. 4.4 (Euler equations): Roe-averaged characteristic decomposition,
//     Rusanov (local Lax-Friedrichs) flux splitting, the split characteristic
//     fluxes as MLP inputs, dimension-by-dimension sweeps (x then y) and the
//     third-order SSP Runge-Kutta scheme.
//
// Arithmetic order.  Every operation below is written out in one fixed order
// (fma only where written, left-to-right otherwise) and this file is compiled
// with -ffp-contract=off, so a*b+c is never contracted behind our back.  That
// makes the oracle a deterministic function of its inputs on any IEEE-754
// machine.
//
// Readings of the paper where it is silent:
//   - negative-side stencil: the mirror image about x_{i+1/2},
//     (g-_{i+3}, ..., g-_{i-2}), through the same network and coefficients;
//   - first-order upwind fallback: g+_{m,i} for the "+" side, g-_{m,i+1} for
//     the "-" side;
//   - LLF alpha_m: max over the six stencil cells of |lambda_m|, first index
//     wins ties;
//   - Roe eigenvectors in the textbook (Toro) scaling;
//   - cell-centred grid, ghost cells by periodic wrap or zero-gradient copy.
//
// Forward-mode derivatives.  The Euler part is a template on the scalar type;
// instantiated with Dual it gives J*v of the right-hand side with the
// classifier mask and the alpha argmax frozen, which the tests use to check the
// CUDA adjoint by the dot-product identity <lambda, J v> = <J^T lambda, v>.

#ifdef _OPENMP
#include <omp.h>
#endif
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual fma(Dual a, Dual b, Dual c) {
  return Dual(std::fma(a.v, b.v, c.v), a.d * b.v + a.v * b.d + c.d);
}
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
inline double val(Dual a) { return a.v; }

inline double fma(double a, double b, double c) { return std::fma(a, b, c); }
inline double sqrt(double a) { return std::sqrt(a); }
inline double fabs(double a) { return std::fabs(a); }
inline double val(double a) { return a; }

// ---------------------------------------------------------------- parameters
}  // namespace

extern "C" {

// Mirrors oracle/__init__.py's ctypes structure field by field.
struct OracleParams {
  int ndim;         // 1 or 2
  int nx, ny;       // interior cells (ny = 1 in 1D)
  int bc_x, bc_y;   // 0 = periodic, 1 = transmissive (zero-gradient)
  int mask_mode;    // 0 = MLP, 1 = all smooth, 2 = all discarded, 3 = given,
                    // 4 = TENO6-opt selection
  int n_layers;     // affine layers of the classifier (5 for 6-64-32-16-8-4)
  int widths[8];    // widths[0] = 6 inputs ... widths[n_layers] = 4 outputs
  double dx, dy, gamma;
  double d[4];        // optimal linear weights d_0..d_3
  double cand[4][4];  // candidate coefficients; S0..S2 use the first three
  const double* net;  // per layer: W[out][in] row-major, then b[out]
  // TENO6-opt smoothness indicators (mask_mode 4): beta = v^T B v with B for
  // S0, S1, S2 (3 x 3 each), S3 (4 x 4), the full stencil (6 x 6), row-major,
  // 79 values; v = the stencil's values minus its first value
  const double* teno;
};

}  // extern "C"

namespace {

enum { MASK_MLP = 0, MASK_SMOOTH = 1, MASK_ROUGH = 2, MASK_GIVEN = 3, MASK_TENO = 4 };

// ------------------------------------------------------ Sec. 3.1 classifier
// Eq. (normalizainput) then Eqs. (reconstuction)/(activationfunction); returns
// eta bits (bit k set <=> stencil S_k discarded, i.e. logit_k > 0).
unsigned classify6(const OracleParams& P, const double s[6], double* logits_out) {
  // Eq. (normalizainput): divide by max(|s_0|, ..., |s_5|, 1).
  double m = 1.0;
  for (int j = 0; j < 6; ++j) m = std::fmax(m, std::fabs(s[j]));
  double x[64], y[64];
  int width_in = P.widths[0];
  for (int j = 0; j < 6; ++j) x[j] = s[j] / m;
  // Eq. (reconstuction): Y^l = w^l X^{l-1} + b^l, each output an fma chain
  // over the inputs in ascending order, started from the bias.
  const double* p = P.net;
  for (int l = 0; l < P.n_layers; ++l) {
    int nin = P.widths[l], nout = P.widths[l + 1];
    const double* W = p;
    const double* b = p + (size_t)nout * nin;
    for (int o = 0; o < nout; ++o) {
      double acc = b[o];
      for (int i = 0; i < nin; ++i) acc = std::fma(W[(size_t)o * nin + i], x[i], acc);
      y[o] = acc;
    }
    p = b + nout;
    bool last = (l == P.n_layers - 1);
    for (int o = 0; o < nout; ++o) {
      // Eq. (activationfunction): ReLU max(x, 0) on hidden layers.
      x[o] = last ? y[o] : (y[o] > 0.0 ? y[o] : 0.0);
    }
    width_in = nout;
  }
  (void)width_in;
  // Eq. (sigmoidfunction) + the 50 % rule: sigmoid(z) > 1/2 <=> z > 0.
  unsigned eta = 0;
  for (int k = 0; k < 4; ++k) {
    if (logits_out) logits_out[k] = x[k];
    if (x[k] > 0.0) eta |= 1u << k;
  }
  return eta;
}

// -------------------------------------------- Sec. 2.1-2.2 TENO6-opt selection
// beta = v^T B v (an integral of squared derivatives: a value that rounds
// below 0 is 0), summed row by row in index order.
double quad_form(const double* B, const double* v, int r) {
  double s = 0.0;
  for (int i = 0; i < r; ++i) {
    double row = 0.0;
    for (int j = 0; j < r; ++j) row = row + B[i * r + j] * v[j];
    s = s + v[i] * row;
  }
  return s > 0.0 ? s : 0.0;
}

// TENO6-opt stencil selection on the six values s (i-2..i+3), returned as
// eta bits (bit k set <=> S_k discarded):
//   beta_k of S0..S3 and beta_6 of the full stencil (Jiang-Shu definition);
//   tau_6 = |beta_6 - (beta_1 + beta_2 + 4 beta_0) / 6|    Eq. (taukTENO)
//   gamma_k = (C + tau_6 / (beta_k + eps))^q, C = 1, q = 6, eps = 1e-40
//                                                          Eq. (measureTENO)
//   chi_k = gamma_k / sum gamma                            Eq. (normalize)
//   delta_k = [chi_k >= C_T], C_T = 1e-6                   Eq. (cut-off)
// gamma_k / gamma_max = (a_k / a_max)^6 with a_k = C + tau_6 / (beta_k + eps)
// (three multiplications) replaces gamma_k in the ratio chi_k: the same
// quotient, without overflow when some beta_k is 0.
unsigned teno6_eta(const OracleParams& P, const double s[6]) {
  static const int cells[4][4] = {{1, 2, 3, 0}, {2, 3, 4, 0}, {0, 1, 2, 0}, {2, 3, 4, 5}};
  const double* B3 = P.teno;
  const double* B4 = P.teno + 27;
  const double* B6 = P.teno + 43;
  double beta[4], v[6];
  for (int k = 0; k < 3; ++k) {
    for (int j = 0; j < 3; ++j) v[j] = s[cells[k][j]] - s[cells[k][0]];
    beta[k] = quad_form(B3 + 9 * k, v, 3);
  }
  for (int j = 0; j < 4; ++j) v[j] = s[cells[3][j]] - s[cells[3][0]];
  beta[3] = quad_form(B4, v, 4);
  for (int j = 0; j < 6; ++j) v[j] = s[j] - s[0];
  const double beta6 = quad_form(B6, v, 6);
  double t = beta[1] + beta[2];
  t = t + 4.0 * beta[0];
  t = t / 6.0;
  const double tau = std::fabs(beta6 - t);
  double a[4], amax = 0.0;
  for (int k = 0; k < 4; ++k) {
    a[k] = 1.0 + tau / (beta[k] + 1e-40);
    amax = k == 0 ? a[k] : std::fmax(amax, a[k]);
  }
  double g[4], sum = 0.0;
  for (int k = 0; k < 4; ++k) {
    const double b = a[k] / amax;
    const double b2 = b * b;
    const double b3 = b2 * b;
    g[k] = b3 * b3;
    sum = sum + g[k];
  }
  unsigned eta = 0;
  for (int k = 0; k < 4; ++k)
    if (!(g[k] / sum >= 1e-6)) eta |= 1u << k;
  return eta;
}

// ----------------------------------------- Sec. 2 + Algorithm 2 reconstruction
// Candidate fluxes on the (un-normalised) six-point stencil s_0..s_5 =
// values at i-2..i+3:  S0 = {i-1,i,i+1}, S1 = {i,i+1,i+2}, S2 = {i-2,i-1,i},
// S3 = {i,i+1,i+2,i+3} (three 3-point stencils and one 4-point stencil of
// incremental width, Fig. 1).
template <class T>
void candidates(const OracleParams& P, const T s[6], T f[4]) {
  static const int first[4] = {1, 2, 0, 2};
  static const int npts[4] = {3, 3, 3, 4};
  for (int k = 0; k < 4; ++k) {
    T acc = T(P.cand[k][0]) * s[first[k]];
    for (int l = 1; l < npts[k]; ++l) acc = fma(T(P.cand[k][l]), s[first[k] + l], acc);
    f[k] = acc;
  }
}

// Eqs. (TENOweight_renormalize) and (convex), with the first-order fallback
// of Algorithm 2 when every stencil is discarded.
template <class T>
T combine(const OracleParams& P, const T s[6], unsigned eta) {
  T f[4];
  candidates(P, s, f);
  double D = 0.0;
  for (int k = 0; k < 4; ++k)
    if (!((eta >> k) & 1u)) D = D + P.d[k];
  if (D == 0.0) return s[2];  // first-order upwind: the stencil's own cell i
  T g = T(0.0);
  for (int k = 0; k < 4; ++k)
    if (!((eta >> k) & 1u)) g = fma(T(P.d[k] / D), f[k], g);
  return g;
}

// ------------------------------------------------------- Sec. 4.4 Euler parts
template <class T>
struct Cell {
  T U[4];   // conserved variables
  T F[4];   // physical flux in the sweep direction
  T un;     // velocity normal to the face
  T u, v;   // velocity components
  T c;      // sound speed
  T H;      // total enthalpy
  T sr;     // sqrt(rho)
};

// Primitive variables and the physical flux of one cell (dir 0 = x, 1 = y).
template <class T>
void cell_state(const OracleParams& P, int dir, const T* U, Cell<T>& o) {
  const int nv = P.ndim == 2 ? 4 : 3;
  const double gm1 = P.gamma - 1.0;
  for (int n = 0; n < nv; ++n) o.U[n] = U[n];
  T rho = U[0];
  T E = U[nv - 1];
  T u = U[1] / rho;
  T v = T(0.0);
  T q;
  if (nv == 4) {
    v = U[2] / rho;
    q = fma(v, v, u * u);
  } else {
    q = u * u;
  }
  T p = T(gm1) * (E - T(0.5) * (rho * q));
  T c = sqrt((T(P.gamma) * p) / rho);
  T Ep = E + p;
  o.u = u;
  o.v = v;
  o.c = c;
  o.H = Ep / rho;
  o.sr = sqrt(rho);
  if (nv == 3) {
    o.un = u;
    o.F[0] = U[1];
    o.F[1] = fma(U[1], u, p);
    o.F[2] = Ep * u;
  } else if (dir == 0) {
    o.un = u;
    o.F[0] = U[1];
    o.F[1] = fma(U[1], u, p);
    o.F[2] = U[2] * u;
    o.F[3] = Ep * u;
  } else {
    o.un = v;
    o.F[0] = U[2];
    o.F[1] = U[1] * v;
    o.F[2] = fma(U[2], v, p);
    o.F[3] = Ep * v;
  }
}

// Roe average of cells a (left) and b (right) and the left/right eigenvector
// matrices of the Roe-averaged flux Jacobian in direction dir.  L[m][n] is
// row m of L (the m-th left eigenvector); R[n][m] is component n of the m-th
// right eigenvector, so that L R = I.
// Field order: 2D (u_n - c, entropy, shear, u_n + c); 1D (u - c, entropy, u + c).
template <class T>
bool roe_eigen(const OracleParams& P, int dir, const Cell<T>& a, const Cell<T>& b,
               T L[4][4], T R[4][4]) {
  const int nv = P.ndim == 2 ? 4 : 3;
  const double gm1 = P.gamma - 1.0;
  T den = a.sr + b.sr;
  T ut = fma(b.sr, b.u, a.sr * a.u) / den;
  T Ht = fma(b.sr, b.H, a.sr * a.H) / den;
  T vt = T(0.0), qt;
  if (nv == 4) {
    vt = fma(b.sr, b.v, a.sr * a.v) / den;
    qt = fma(vt, vt, ut * ut);
  } else {
    qt = ut * ut;
  }
  T c2 = T(gm1) * (Ht - T(0.5) * qt);
  bool ok = val(c2) > 0.0;
  T ct = sqrt(c2);
  T ic = T(1.0) / ct;
  T b1 = T(gm1) / c2;
  T b2 = T(0.5) * (b1 * qt);
  T nt = (nv == 4 && dir == 1) ? vt : ut;  // normal Roe velocity
  T nc = nt * ic;
  T b1u = b1 * ut;
  T b1v = b1 * vt;
  T hb1 = T(0.5) * b1;
  T ntc = nt * ct;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) L[m][n] = R[m][n] = T(0.0);
  if (nv == 3) {
    L[0][0] = T(0.5) * (b2 + nc);
    L[0][1] = T(0.5) * (-b1u - ic);
    L[0][2] = hb1;
    L[1][0] = T(1.0) - b2;
    L[1][1] = b1u;
    L[1][2] = -b1;
    L[2][0] = T(0.5) * (b2 - nc);
    L[2][1] = T(0.5) * (-b1u + ic);
    L[2][2] = hb1;
    // columns: (1, u-c, H-uc), (1, u, q/2), (1, u+c, H+uc)
    R[0][0] = T(1.0);  R[0][1] = T(1.0);           R[0][2] = T(1.0);
    R[1][0] = ut - ct; R[1][1] = ut;               R[1][2] = ut + ct;
    R[2][0] = Ht - ntc; R[2][1] = T(0.5) * qt;     R[2][2] = Ht + ntc;
    return ok;
  }
  if (dir == 0) {
    L[0][0] = T(0.5) * (b2 + nc);
    L[0][1] = T(0.5) * (-b1u - ic);
    L[0][2] = T(0.5) * (-b1v);
    L[0][3] = hb1;
    L[1][0] = T(1.0) - b2;
    L[1][1] = b1u;
    L[1][2] = b1v;
    L[1][3] = -b1;
    L[2][0] = -vt;
    L[2][1] = T(0.0);
    L[2][2] = T(1.0);
    L[2][3] = T(0.0);
    L[3][0] = T(0.5) * (b2 - nc);
    L[3][1] = T(0.5) * (-b1u + ic);
    L[3][2] = T(0.5) * (-b1v);
    L[3][3] = hb1;
    // columns: (1,u-c,v,H-uc), (1,u,v,q/2), (0,0,1,v), (1,u+c,v,H+uc)
    R[0][0] = T(1.0);   R[0][1] = T(1.0);       R[0][2] = T(0.0); R[0][3] = T(1.0);
    R[1][0] = ut - ct;  R[1][1] = ut;           R[1][2] = T(0.0); R[1][3] = ut + ct;
    R[2][0] = vt;       R[2][1] = vt;           R[2][2] = T(1.0); R[2][3] = vt;
    R[3][0] = Ht - ntc; R[3][1] = T(0.5) * qt;  R[3][2] = vt;     R[3][3] = Ht + ntc;
  } else {
    L[0][0] = T(0.5) * (b2 + nc);
    L[0][1] = T(0.5) * (-b1u);
    L[0][2] = T(0.5) * (-b1v - ic);
    L[0][3] = hb1;
    L[1][0] = T(1.0) - b2;
    L[1][1] = b1u;
    L[1][2] = b1v;
    L[1][3] = -b1;
    L[2][0] = -ut;
    L[2][1] = T(1.0);
    L[2][2] = T(0.0);
    L[2][3] = T(0.0);
    L[3][0] = T(0.5) * (b2 - nc);
    L[3][1] = T(0.5) * (-b1u);
    L[3][2] = T(0.5) * (-b1v + ic);
    L[3][3] = hb1;
    // columns: (1,u,v-c,H-vc), (1,u,v,q/2), (0,1,0,u), (1,u,v+c,H+vc)
    R[0][0] = T(1.0);   R[0][1] = T(1.0);       R[0][2] = T(0.0); R[0][3] = T(1.0);
    R[1][0] = ut;       R[1][1] = ut;           R[1][2] = T(1.0); R[1][3] = ut;
    R[2][0] = vt - ct;  R[2][1] = vt;           R[2][2] = T(0.0); R[2][3] = vt + ct;
    R[3][0] = Ht - ntc; R[3][1] = T(0.5) * qt;  R[3][2] = ut;     R[3][3] = Ht + ntc;
  }
  return ok;
}

// |lambda_m| of a cell: 2D (u_n - c, u_n, u_n, u_n + c), 1D (u - c, u, u + c).
template <class T>
T abs_lambda(int nv, int m, const Cell<T>& c) {
  if (m == 0) return fabs(c.un - c.c);
  if (m == nv - 1) return fabs(c.un + c.c);
  return fabs(c.un);
}

// One face F_{i+1/2} from the six stencil cells st[0..5] = cells i-2..i+3.
// eta_io: per field m, byte (eta+ | eta- << 4); read when the mode is "given",
// written otherwise (may be null when not given).  Returns false when the
// state is non-physical (Roe sound speed squared <= 0).
template <class T>
bool face_flux(const OracleParams& P, int dir, const Cell<T> st[6], uint8_t* eta_io,
               T Fhat[4]) {
  const int nv = P.ndim == 2 ? 4 : 3;
  T L[4][4], R[4][4];
  bool ok = roe_eigen(P, dir, st[2], st[3], L, R);
  T gh[4];
  for (int m = 0; m < nv; ++m) {
    // Rusanov / local Lax-Friedrichs: alpha_m = max_j |lambda_m(U_j)|.
    T alpha = abs_lambda(nv, m, st[0]);
    for (int j = 1; j < 6; ++j) {
      T a = abs_lambda(nv, m, st[j]);
      if (val(a) > val(alpha)) alpha = a;
    }
    // Characteristic projection and splitting g+-_{m,j} = (g + - alpha v) / 2.
    T sp[6], sm[6];
    for (int j = 0; j < 6; ++j) {
      T vv = L[m][0] * st[j].U[0];
      T gg = L[m][0] * st[j].F[0];
      for (int n = 1; n < nv; ++n) {
        vv = fma(L[m][n], st[j].U[n], vv);
        gg = fma(L[m][n], st[j].F[n], gg);
      }
      sp[j] = T(0.5) * fma(alpha, vv, gg);
      sm[j] = T(0.5) * fma(-alpha, vv, gg);
    }
    // The "-" side is the mirror image of the "+" side about x_{i+1/2}.
    T sneg[6];
    for (int j = 0; j < 6; ++j) sneg[j] = sm[5 - j];
    unsigned ep, em;
    if (P.mask_mode == MASK_GIVEN) {
      ep = eta_io[m] & 15u;
      em = (eta_io[m] >> 4) & 15u;
    } else if (P.mask_mode == MASK_SMOOTH) {
      ep = em = 0u;
    } else if (P.mask_mode == MASK_ROUGH) {
      ep = em = 15u;
    } else {
      double xp[6], xm[6];
      for (int j = 0; j < 6; ++j) {
        xp[j] = val(sp[j]);
        xm[j] = val(sneg[j]);
      }
      if (P.mask_mode == MASK_TENO) {
        ep = teno6_eta(P, xp);
        em = teno6_eta(P, xm);
      } else {
        ep = classify6(P, xp, nullptr);
        em = classify6(P, xm, nullptr);
      }
    }
    if (eta_io && P.mask_mode != MASK_GIVEN) eta_io[m] = (uint8_t)(ep | (em << 4));
    T gp = combine(P, sp, ep);
    T gm = combine(P, sneg, em);
    gh[m] = gp + gm;
  }
  // Back to physical space: F_n = sum_m R[n][m] gh_m.
  for (int n = 0; n < nv; ++n) {
    T acc = R[n][0] * gh[0];
    for (int m = 1; m < nv; ++m) acc = fma(R[n][m], gh[m], acc);
    Fhat[n] = acc;
  }
  return ok;
}

// ------------------------------------------------------------ grid handling
inline int ghost(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

template <class T>
void load_cell(const OracleParams& P, const T* U, int i, int j, T* out) {
  const int nv = P.ndim == 2 ? 4 : 3;
  size_t plane = (size_t)P.nx * P.ny;
  size_t idx = (size_t)j * P.nx + i;
  for (int n = 0; n < nv; ++n) out[n] = U[n * plane + idx];
}

// Face f (0..nx) of row j in x, or face f (0..ny) of column i in y: the face
// between cells f-1 and f; its stencil is cells f-3..f+2.
template <class T>
bool face_at(const OracleParams& P, const T* U, int dir, int f, int line, uint8_t* eta_io,
             T Fhat[4]) {
  Cell<T> st[6];
  T cu[4];
  for (int k = 0; k < 6; ++k) {
    if (dir == 0)
      load_cell(P, U, ghost(f - 3 + k, P.nx, P.bc_x), line, cu);
    else
      load_cell(P, U, line, ghost(f - 3 + k, P.ny, P.bc_y), cu);
    cell_state(P, dir, cu, st[k]);
  }
  return face_flux(P, dir, st, eta_io, Fhat);
}

inline size_t mask_x_index(const OracleParams& P, int m, int j, int f) {
  return ((size_t)m * P.ny + j) * (P.nx + 1) + f;
}
inline size_t mask_y_index(const OracleParams& P, int m, int j, int i) {
  const int nv = P.ndim == 2 ? 4 : 3;
  size_t xblock = (size_t)nv * P.ny * (P.nx + 1);
  return xblock + ((size_t)m * (P.ny + 1) + j) * P.nx + i;
}

// The semi-discrete right-hand side: x sweep, then y sweep, then the
// conservative difference -(F_{i+1/2}-F_{i-1/2})/dx - (G_{j+1/2}-G_{j-1/2})/dy.
template <class T>
int rhs_impl(const OracleParams& P, const T* U, T* dUdt, const uint8_t* mask_in,
             uint8_t* mask_out) {
  const int nv = P.ndim == 2 ? 4 : 3;
  const int nx = P.nx, ny = P.ny;
  int bad = 0;
  std::vector<T> Fx((size_t)ny * (nx + 1) * nv);
  std::vector<T> Fy(P.ndim == 2 ? (size_t)(ny + 1) * nx * nv : 0);
  // Faces are independent: with OpenMP the lines of faces are shared among
  // threads; every face's arithmetic, and where its result goes, is the
  // same as in a serial run.
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int j = 0; j < ny; ++j)
    for (int f = 0; f <= nx; ++f) {
      uint8_t eta[4] = {0, 0, 0, 0};
      if (P.mask_mode == MASK_GIVEN)
        for (int m = 0; m < nv; ++m) eta[m] = mask_in[mask_x_index(P, m, j, f)];
      if (!face_at(P, U, 0, f, j, eta, &Fx[((size_t)j * (nx + 1) + f) * nv])) bad = 1;
      if (mask_out)
        for (int m = 0; m < nv; ++m) mask_out[mask_x_index(P, m, j, f)] = eta[m];
    }
  if (P.ndim == 2) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int f = 0; f <= ny; ++f)
      for (int i = 0; i < nx; ++i) {
        uint8_t eta[4] = {0, 0, 0, 0};
        if (P.mask_mode == MASK_GIVEN)
          for (int m = 0; m < nv; ++m) eta[m] = mask_in[mask_y_index(P, m, f, i)];
        if (!face_at(P, U, 1, f, i, eta, &Fy[((size_t)f * nx + i) * nv])) bad = 1;
        if (mask_out)
          for (int m = 0; m < nv; ++m) mask_out[mask_y_index(P, m, f, i)] = eta[m];
      }
  }
  size_t plane = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int n = 0; n < nv; ++n) {
        T Fp = Fx[((size_t)j * (nx + 1) + i + 1) * nv + n];
        T Fm = Fx[((size_t)j * (nx + 1) + i) * nv + n];
        T r = -((Fp - Fm) / T(P.dx));
        if (P.ndim == 2) {
          T Gp = Fy[((size_t)(j + 1) * nx + i) * nv + n];
          T Gm = Fy[((size_t)j * nx + i) * nv + n];
          r = r - (Gp - Gm) / T(P.dy);
        }
        dUdt[n * plane + (size_t)j * nx + i] = r;
      }
  return bad;
}

}  // namespace

extern "C" {

// Threads of the face loops (OpenMP builds; 1 otherwise): sets the count for
// later calls (n >= 1) and returns the count in force.
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// dU/dt of the whole grid.  U, dUdt: [nv][ny][nx] FP64.  mask_in is read when
// mask_mode == 3; mask_out (nullable) receives the classifier bits, layout
// x faces [nv][ny][nx+1] then y faces [nv][ny+1][nx].  Returns 1 if any Roe
// state was non-physical, else 0.
int oracle_rhs(const OracleParams* P, const double* U, double* dUdt, const uint8_t* mask_in,
               uint8_t* mask_out) {
  return rhs_impl<double>(*P, U, dUdt, mask_in, mask_out);
}

// dU/dt at a list of cells only (flat indices j*nx+i); out is [ncells][nv].
// Each cell evaluates its own two (four in 2D) faces with exactly the code
// above, so the values are bit-identical to oracle_rhs.
int oracle_rhs_cells(const OracleParams* P, const double* U, int64_t ncells,
                     const int64_t* cells, double* out) {
  const int nv = P->ndim == 2 ? 4 : 3;
  int bad = 0;
  for (int64_t c = 0; c < ncells; ++c) {
    int i = (int)(cells[c] % P->nx), j = (int)(cells[c] / P->nx);
    double Fp[4], Fm[4], Gp[4], Gm[4];
    uint8_t eta[4];
    if (P->mask_mode == MASK_GIVEN) return -1;
    if (!face_at(*P, U, 0, i + 1, j, eta, Fp)) bad = 1;
    if (!face_at(*P, U, 0, i, j, eta, Fm)) bad = 1;
    if (P->ndim == 2) {
      if (!face_at(*P, U, 1, j + 1, i, eta, Gp)) bad = 1;
      if (!face_at(*P, U, 1, j, i, eta, Gm)) bad = 1;
    }
    for (int n = 0; n < nv; ++n) {
      double r = -((Fp[n] - Fm[n]) / P->dx);
      if (P->ndim == 2) r = r - (Gp[n] - Gm[n]) / P->dy;
      out[c * nv + n] = r;
    }
  }
  return bad;
}

// Face masks of a list of faces: dir 0/1, face index f and line index
// (row j for x faces, column i for y faces); out[k*nv + m] = eta byte.
int oracle_face_masks(const OracleParams* P, const double* U, int64_t nfaces,
                      const int32_t* dir, const int32_t* f, const int32_t* line, uint8_t* out) {
  const int nv = P->ndim == 2 ? 4 : 3;
  if (P->mask_mode == MASK_GIVEN) return -1;
  double Fh[4];
  int bad = 0;
  for (int64_t k = 0; k < nfaces; ++k)
    if (!face_at(*P, U, dir[k], f[k], line[k], out + k * nv, Fh)) bad = 1;
  return bad;
}

// J v of the right-hand side (forward mode), the mask frozen to mask_in and the
// alpha argmax frozen at the primal state.  dUdt (nullable) receives the
// primal values.
int oracle_rhs_jvp(const OracleParams* P, const double* U, const double* V,
                   const uint8_t* mask_in, double* dUdt, double* JV) {
  const int nv = P->ndim == 2 ? 4 : 3;
  size_t n = (size_t)nv * P->nx * P->ny;
  std::vector<Dual> Ud(n), Rd(n);
  for (size_t k = 0; k < n; ++k) Ud[k] = Dual(U[k], V[k]);
  OracleParams Q = *P;
  Q.mask_mode = MASK_GIVEN;
  int bad = rhs_impl<Dual>(Q, Ud.data(), Rd.data(), mask_in, nullptr);
  for (size_t k = 0; k < n; ++k) {
    if (dUdt) dUdt[k] = Rd[k].v;
    JV[k] = Rd[k].d;
  }
  return bad;
}

// J v of the right-hand side at a list of cells only (flat indices j*nx+i),
// mask frozen to mask_in, alpha argmax frozen at the primal state; out is
// [ncells][nv].  Each cell evaluates its own two (four in 2D) faces with the
// dual-number code of oracle_rhs_jvp, the stencil cells loaded as (U, V).
int oracle_rhs_jvp_cells(const OracleParams* P, const double* U, const double* V,
                         const uint8_t* mask_in, int64_t ncells, const int64_t* cells, double* out) {
  const int nv = P->ndim == 2 ? 4 : 3;
  OracleParams Q = *P;
  Q.mask_mode = MASK_GIVEN;
  const size_t plane = (size_t)Q.nx * Q.ny;
  auto face = [&](int dir, int f, int line, Dual Fh[4]) {
    Cell<Dual> st[6];
    Dual cu[4];
    for (int k = 0; k < 6; ++k) {
      const int i = dir == 0 ? ghost(f - 3 + k, Q.nx, Q.bc_x) : line;
      const int j = dir == 0 ? line : ghost(f - 3 + k, Q.ny, Q.bc_y);
      const size_t idx = (size_t)j * Q.nx + i;
      for (int n = 0; n < nv; ++n) cu[n] = Dual(U[n * plane + idx], V[n * plane + idx]);
      cell_state(Q, dir, cu, st[k]);
    }
    uint8_t eta[4] = {0, 0, 0, 0};
    for (int m = 0; m < nv; ++m)
      eta[m] = mask_in[dir == 0 ? mask_x_index(Q, m, line, f) : mask_y_index(Q, m, f, line)];
    return face_flux(Q, dir, st, eta, Fh);
  };
  int bad = 0;
  for (int64_t c = 0; c < ncells; ++c) {
    const int i = (int)(cells[c] % Q.nx), j = (int)(cells[c] / Q.nx);
    Dual Fp[4], Fm[4], Gp[4], Gm[4];
    if (!face(0, i + 1, j, Fp)) bad = 1;
    if (!face(0, i, j, Fm)) bad = 1;
    if (Q.ndim == 2) {
      if (!face(1, j + 1, i, Gp)) bad = 1;
      if (!face(1, j, i, Gm)) bad = 1;
    }
    for (int n = 0; n < nv; ++n) {
      Dual r = -((Fp[n] - Fm[n]) / Dual(Q.dx));
      if (Q.ndim == 2) r = r - (Gp[n] - Gm[n]) / Dual(Q.dy);
      out[c * nv + n] = r.d;
    }
  }
  return bad;
}

// Sec. 3.1 classifier alone: X [n][6] raw stencil values -> eta bits (and the
// four logits when logits != null).
int oracle_classify(const OracleParams* P, const double* X, int64_t n, uint8_t* eta,
                    double* logits) {
  for (int64_t r = 0; r < n; ++r)
    eta[r] = (uint8_t)classify6(*P, X + r * 6, logits ? logits + r * 4 : nullptr);
  return 0;
}

// One scalar six-point reconstruction (Algorithm 2 on one stencil):
// returns the reconstructed value; eta_io as in face_flux (low nibble only).
double oracle_reconstruct(const OracleParams* P, const double s[6], uint8_t* eta_io) {
  unsigned eta;
  if (P->mask_mode == MASK_GIVEN)
    eta = *eta_io & 15u;
  else if (P->mask_mode == MASK_SMOOTH)
    eta = 0u;
  else if (P->mask_mode == MASK_ROUGH)
    eta = 15u;
  else if (P->mask_mode == MASK_TENO)
    eta = teno6_eta(*P, s);
  else
    eta = classify6(*P, s, nullptr);
  if (eta_io) *eta_io = (uint8_t)eta;
  return combine(*P, s, eta);
}

// Roe eigenvector matrices between two cell states (tests: L R = I).
int oracle_roe_eigen(const OracleParams* P, int dir, const double* UL, const double* UR,
                     double* L, double* R) {
  Cell<double> a, b;
  cell_state(*P, dir, UL, a);
  cell_state(*P, dir, UR, b);
  double l[4][4], r[4][4];
  bool ok = roe_eigen(*P, dir, a, b, l, r);
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) {
      L[m * 4 + n] = l[m][n];
      R[m * 4 + n] = r[m][n];
    }
  return ok ? 0 : 1;
}

// Time step of Sec. 4.4's SSP-RK3 from the state U^n:
// dt = cfl / (max(|u|+c)/dx + max(|v|+c)/dy)  (1D: cfl / (max(|u|+c)/dx)).
double oracle_dt(const OracleParams* P, const double* U, double cfl) {
  const int nv = P->ndim == 2 ? 4 : 3;
  double sx = 0.0, sy = 0.0;
  double cu[4];
  for (int j = 0; j < P->ny; ++j)
    for (int i = 0; i < P->nx; ++i) {
      load_cell(*P, U, i, j, cu);
      Cell<double> c;
      cell_state(*P, 0, cu, c);
      sx = std::fmax(sx, std::fabs(c.u) + c.c);
      if (nv == 4) sy = std::fmax(sy, std::fabs(c.v) + c.c);
    }
  double a = sx / P->dx;
  if (nv == 4) a = a + sy / P->dy;
  return cfl / a;
}

// One third-order SSP Runge-Kutta step (Gottlieb & Shu form):
//   U1 = U + dt L(U)
//   U2 = 3/4 U + 1/4 (U1 + dt L(U1))
//   U  = 1/3 U + 2/3 (U2 + dt L(U2))
// dt from oracle_dt, clipped so that t + dt <= t_end when t_end > 0.
// *t is advanced; *dt_out (nullable) receives dt.
int oracle_step(const OracleParams* P, double* U, double cfl, double* t, double t_end,
                double* dt_out) {
  const int nv = P->ndim == 2 ? 4 : 3;
  size_t n = (size_t)nv * P->nx * P->ny;
  double dt = oracle_dt(P, U, cfl);
  if (t_end > 0.0 && *t + dt > t_end) dt = t_end - *t;
  std::vector<double> L(n), U1(n), U2(n);
  int bad = rhs_impl<double>(*P, U, L.data(), nullptr, nullptr);
  for (size_t k = 0; k < n; ++k) U1[k] = std::fma(dt, L[k], U[k]);
  bad |= rhs_impl<double>(*P, U1.data(), L.data(), nullptr, nullptr);
  for (size_t k = 0; k < n; ++k) U2[k] = std::fma(0.75, U[k], 0.25 * std::fma(dt, L[k], U1[k]));
  bad |= rhs_impl<double>(*P, U2.data(), L.data(), nullptr, nullptr);
  const double third = 1.0 / 3.0, two_thirds = 2.0 / 3.0;
  for (size_t k = 0; k < n; ++k)
    U[k] = std::fma(third, U[k], two_thirds * std::fma(dt, L[k], U2[k]));
  *t = *t + dt;
  if (dt_out) *dt_out = dt;
  return bad;
}

// Scalar conservation law u_t + f(u)_x = 0 on a periodic 1D grid (Sec. 4.1,
// 4.2): law 0 = linear advection f = u, law 1 = Burgers f = u^2/2.  Local
// Lax-Friedrichs split with alpha = max over the stencil of |f'(u)|, the same
// six-point reconstruction (mirrored for the "-" side), SSP-RK3 with a fixed
// dt = cfl*dx/max|f'| of the initial data, run to t_end (last step clipped).
static void scalar_rhs(const OracleParams& P, int law, const std::vector<double>& u,
                       std::vector<double>& dudt, std::vector<double>& F) {
  const int n = P.nx;
  for (int f = 0; f <= n; ++f) {
    double uu[6], fl[6];
    for (int k = 0; k < 6; ++k) {
      uu[k] = u[ghost(f - 3 + k, n, P.bc_x)];
      fl[k] = law == 0 ? uu[k] : 0.5 * (uu[k] * uu[k]);
    }
    double alpha = law == 0 ? 1.0 : std::fabs(uu[0]);
    if (law == 1)
      for (int k = 1; k < 6; ++k) alpha = std::fmax(alpha, std::fabs(uu[k]));
    double sp[6], sm[6], sneg[6];
    for (int k = 0; k < 6; ++k) {
      sp[k] = 0.5 * std::fma(alpha, uu[k], fl[k]);
      sm[k] = 0.5 * std::fma(-alpha, uu[k], fl[k]);
    }
    for (int k = 0; k < 6; ++k) sneg[k] = sm[5 - k];
    unsigned ep, em;
    if (P.mask_mode == MASK_SMOOTH) ep = em = 0u;
    else if (P.mask_mode == MASK_ROUGH) ep = em = 15u;
    else if (P.mask_mode == MASK_TENO) {
      ep = teno6_eta(P, sp);
      em = teno6_eta(P, sneg);
    } else {
      ep = classify6(P, sp, nullptr);
      em = classify6(P, sneg, nullptr);
    }
    F[f] = combine(P, sp, ep) + combine(P, sneg, em);
  }
  for (int i = 0; i < n; ++i) dudt[i] = -((F[i + 1] - F[i]) / P.dx);
}

int oracle_scalar_solve(const OracleParams* P, int law, double* u0, double cfl, double t_end,
                        int64_t* nsteps_out) {
  const int n = P->nx;
  std::vector<double> u(u0, u0 + n), L(n), u1(n), u2(n), F(n + 1);
  double amax = 0.0;
  for (int i = 0; i < n; ++i) amax = std::fmax(amax, law == 0 ? 1.0 : std::fabs(u[i]));
  double dt = cfl * P->dx / amax;
  double t = 0.0;
  int64_t steps = 0;
  while (t < t_end) {
    double h = dt;
    if (t + h > t_end) h = t_end - t;
    scalar_rhs(*P, law, u, L, F);
    for (int i = 0; i < n; ++i) u1[i] = std::fma(h, L[i], u[i]);
    scalar_rhs(*P, law, u1, L, F);
    for (int i = 0; i < n; ++i) u2[i] = std::fma(0.75, u[i], 0.25 * std::fma(h, L[i], u1[i]));
    scalar_rhs(*P, law, u2, L, F);
    for (int i = 0; i < n; ++i)
      u[i] = std::fma(1.0 / 3.0, u[i], (2.0 / 3.0) * std::fma(h, L[i], u2[i]));
    t = t + h;
    ++steps;
  }
  for (int i = 0; i < n; ++i) u0[i] = u[i];
  if (nsteps_out) *nsteps_out = steps;
  return 0;
}

}  // extern "C"
