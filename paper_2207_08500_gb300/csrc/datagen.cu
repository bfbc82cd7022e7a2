// Training data of the classifier on the device (Algorithm 1, Table 9, Sec.
// 3.2): one thread per sample turns nine caller-given uniform draws into a
// six-point stencil, its labels and its function family.
//
// Per sample (draw columns 0..8):
//   0     grid N in {50, 100, 200} with probabilities 40 / 40 / 20 % on
//         [-1, 1], cell centres x_j = -1 + (j + 1/2) dx, dx = 2 / N;
//   1     family 1..9 of Table 9, equally likely;
//   2     interface x_{i+1/2}: i uniform in 2..N-4 (stencil i-2..i+3 inside);
//   3..7  the family's parameters (ranges of Table 9, with the readings:
//         family 2 a ~ U[0.1, 2]; family 5 b1 ~ N(0, 0.6) by Box-Muller;
//         family 6 joins (x-a1)^k1 and (x-a2)^k2, k in 2..8, continuously at
//         x_k ~ U[-0.6, 0.6]; family 8 levels U[-2, 2], jump at the
//         interface for half the samples and at another face inside the
//         stencil for the rest; family 9 N_f ~ U[N/8, N/2]);
//   8     sign: the sample is negated with probability 1/2.
// Labels: families 1-3 none; 4-8 eta_k = 1 iff a singular point lies
// strictly between the outermost cell centres of S_k; family 9 by the
// TENO6-opt selection of Sec. 2 (Eqs. (measureTENO), (taukTENO),
// (normalize), (cut-off); C = 1, q = 6, eps = 1e-40, C_T = 1e-6), with
// smoothness indicators from the Jiang-Shu definition.  Output values are
// normalised by Eq. (normalizainput).
//
// This unit is compiled with -fmad=false and evaluates every expression in
// the order written, so grids, positions and singular points are the exact
// binary64 values of the recipe; the transcendental functions (sin, cos,
// exp, log) are CUDA's and may differ from a host library in the last bit.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace neno6 {
namespace {

constexpr int kDraws = 9;
constexpr int kThreads = 256;

// Smoothness-indicator quadratic forms: beta = v^T B v over the stencil's
// values v (each taken relative to the stencil's first value).
struct TenoTables {
  double b3[3][9];  // S_0 {i-1,i,i+1}, S_1 {i,i+1,i+2}, S_2 {i-2,i-1,i}
  double b4[16];    // S_3 {i..i+3}
  double b6[36];    // the full stencil i-2..i+3
};

// B for cell offsets o[0..r-1] (unit spacing, cell i centred at 0):
// the degree r-1 polynomial with the given cell averages has coefficients
// a = A^-1 v, A_jl = mean of x^l over cell o_j; beta = sum over l = 1..r-1
// of the integral over the central cell of (d^l p / dx^l)^2 = a^T M a.
void beta_matrix(const int* o, int r, double* B) {
  double A[6][12];
  for (int j = 0; j < r; ++j) {
    for (int l = 0; l < r; ++l) {
      const double hi = o[j] + 0.5, lo = o[j] - 0.5;
      A[j][l] = (std::pow(hi, l + 1) - std::pow(lo, l + 1)) / (l + 1);
    }
    for (int l = 0; l < r; ++l) A[j][r + l] = j == l ? 1.0 : 0.0;
  }
  // Gauss-Jordan with partial pivoting: [A | I] -> [I | A^-1]
  for (int c = 0; c < r; ++c) {
    int piv = c;
    for (int j = c + 1; j < r; ++j)
      if (std::fabs(A[j][c]) > std::fabs(A[piv][c])) piv = j;
    if (piv != c)
      for (int l = 0; l < 2 * r; ++l) std::swap(A[c][l], A[piv][l]);
    const double d = A[c][c];
    for (int l = 0; l < 2 * r; ++l) A[c][l] /= d;
    for (int j = 0; j < r; ++j) {
      if (j == c) continue;
      const double f = A[j][c];
      for (int l = 0; l < 2 * r; ++l) A[j][l] -= f * A[c][l];
    }
  }
  // M_pq = sum_l (p!/(p-l)!) (q!/(q-l)!) * integral of x^(p+q-2l) over [-1/2, 1/2]
  auto falling = [](int p, int l) {
    double f = 1.0;
    for (int t = 0; t < l; ++t) f *= (p - t);
    return f;
  };
  double M[6][6] = {};
  for (int p = 0; p < r; ++p)
    for (int q = 0; q < r; ++q)
      for (int l = 1; l < r; ++l) {
        if (l > p || l > q) continue;
        const int m = p + q - 2 * l;
        if (m % 2) continue;
        M[p][q] += falling(p, l) * falling(q, l) * (2.0 * std::pow(0.5, m + 1) / (m + 1));
      }
  // B = (A^-1)^T M A^-1
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      double s = 0.0;
      for (int p = 0; p < r; ++p)
        for (int q = 0; q < r; ++q) s += A[p][r + i] * M[p][q] * A[q][r + j];
      B[i * r + j] = s;
    }
}

const TenoTables& teno_tables() {
  static const TenoTables t = [] {
    TenoTables x{};
    const int s0[3] = {-1, 0, 1}, s1[3] = {0, 1, 2}, s2[3] = {-2, -1, 0}, s3[4] = {0, 1, 2, 3};
    const int full[6] = {-2, -1, 0, 1, 2, 3};
    beta_matrix(s0, 3, x.b3[0]);
    beta_matrix(s1, 3, x.b3[1]);
    beta_matrix(s2, 3, x.b3[2]);
    beta_matrix(s3, 4, x.b4);
    beta_matrix(full, 6, x.b6);
    return x;
  }();
  return t;
}

// positions (0..5 = cells i-2..i+3) of the candidate sub-stencils; the
// outermost cell offsets of S_k are kSpan[k]
__constant__ int kCells[4][4] = {{1, 2, 3, -1}, {2, 3, 4, -1}, {0, 1, 2, -1}, {2, 3, 4, 5}};
__constant__ int kSpan[4][2] = {{-1, 1}, {0, 2}, {-2, 0}, {0, 3}};

__device__ double ipow(double b, int k) {
  double r = b;
  for (int t = 1; t < k; ++t) r = r * b;
  return r;
}

template <int R>
__device__ double quad_form(const double* B, const double* v) {
  double s = 0.0;
  for (int i = 0; i < R; ++i) {
    double row = 0.0;
    for (int j = 0; j < R; ++j) row = row + B[i * R + j] * v[j];
    s = s + v[i] * row;
  }
  return s > 0.0 ? s : 0.0;  // an integral of squares: rounding below 0 is 0
}

// TENO6-opt labels (1 = sub-stencil discarded) of the six values f.
__device__ unsigned teno_labels(const TenoTables& T, const double* f) {
  double beta[4], v[6];
  for (int k = 0; k < 3; ++k) {
    for (int j = 0; j < 3; ++j) v[j] = f[kCells[k][j]] - f[kCells[k][0]];
    beta[k] = quad_form<3>(T.b3[k], v);
  }
  for (int j = 0; j < 4; ++j) v[j] = f[kCells[3][j]] - f[kCells[3][0]];
  beta[3] = quad_form<4>(T.b4, v);
  for (int j = 0; j < 6; ++j) v[j] = f[j] - f[0];
  const double b6 = quad_form<6>(T.b6, v);
  const double tau = fabs(b6 - (beta[1] + beta[2] + 4.0 * beta[0]) / 6.0);
  // gamma_k = (C + tau / (beta_k + eps))^q, normalised: in the log domain
  double lg[4], mx = -INFINITY;
  for (int k = 0; k < 4; ++k) {
    lg[k] = 6.0 * log(1.0 + tau / (beta[k] + 1e-40));
    mx = fmax(mx, lg[k]);
  }
  double g[4], sum = 0.0;
  for (int k = 0; k < 4; ++k) {
    g[k] = exp(lg[k] - mx);
    sum = sum + g[k];
  }
  unsigned eta = 0;
  for (int k = 0; k < 4; ++k)
    if (!(g[k] / sum >= 1e-6)) eta |= 1u << k;
  return eta;
}

__global__ void __launch_bounds__(kThreads) datagen_kernel(const double* __restrict__ u, long long n,
                                                           double* __restrict__ X, uint8_t* __restrict__ labels,
                                                           uint8_t* __restrict__ family, int* status,
                                                           TenoTables T) {
  const double pi = 3.141592653589793;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    double q[kDraws];
    bool ok = true;
    for (int c = 0; c < kDraws; ++c) {
      q[c] = u[r * kDraws + c];
      ok = ok && q[c] >= 0.0 && q[c] < 1.0;
    }
    if (!ok) {
      atomicOr(status, 8);
      for (int j = 0; j < 6; ++j) X[r * 6 + j] = 0.0;
      labels[r] = 0;
      if (family) family[r] = 0;
      continue;
    }
    const int N = q[0] < 0.4 ? 50 : (q[0] < 0.8 ? 100 : 200);
    const int f = 1 + min((int)(9.0 * q[1]), 8);
    const int i = 2 + min((int)((N - 5) * q[2]), N - 6);
    const double* p = q + 3;
    const double dx = 2.0 / N;
    const double xi = -1.0 + (i + 0.5) * dx;
    double x[6], F[6];
    for (int j = 0; j < 6; ++j) x[j] = xi + (j - 2) * dx;
    double sing[2];
    int nsing = 0;
    double period = 0.0;
    if (f == 1) {
      const double k = -5.0 + 10.0 * p[0];
      for (int j = 0; j < 6; ++j) F[j] = k * x[j];
    } else if (f == 2) {
      const double a = 0.1 + 1.9 * p[0], k = 1.0 + 4.0 * p[1];
      for (int j = 0; j < 6; ++j) F[j] = a * sin(k * x[j]);
    } else if (f == 3) {
      const double a1 = -1.0 + 2.0 * p[0], a2 = -1.0 + 2.0 * p[1];
      for (int j = 0; j < 6; ++j) F[j] = exp(a1 * ((x[j] - a2) * (x[j] - a2)));
    } else if (f == 4) {
      const double rr = 1.0 + 2.0 * p[0], P = (2.0 + 6.0 * p[1]) * dx;
      for (int j = 0; j < 6; ++j) {
        const double md = x[j] - (2.0 * P) * floor(x[j] / (2.0 * P));
        F[j] = (rr / P) * (P - fabs(md - P));
      }
      period = P;
    } else if (f == 5) {
      const double b1 = sqrt(0.6) * (sqrt(-2.0 * log(1.0 - p[0])) * cos((2.0 * pi) * p[1]));
      const double x0 = -0.6 + 1.2 * p[2], c = p[3];
      for (int j = 0; j < 6; ++j) F[j] = fmax(0.0, b1 * (x[j] - x0)) + c;
      sing[nsing++] = x0;
    } else if (f == 6) {
      const int k1 = 2 + min((int)(7.0 * p[0]), 6), k2 = 2 + min((int)(7.0 * p[1]), 6);
      const double a1 = 2.0 * p[2], a2 = 2.0 * p[3], xk = -0.6 + 1.2 * p[4];
      const double jump = ipow(xk - a1, k1) - ipow(xk - a2, k2);
      for (int j = 0; j < 6; ++j) F[j] = x[j] <= xk ? ipow(x[j] - a1, k1) : ipow(x[j] - a2, k2) + jump;
      sing[nsing++] = xk;
    } else if (f == 7) {
      const double al = 0.05 + 1.95 * p[0], a = 2.0 * p[1];
      for (int j = 0; j < 6; ++j) F[j] = sqrt(fmax(0.0, 1.0 - (al * al) * ((x[j] - a) * (x[j] - a))));
      sing[nsing++] = a - 1.0 / al;
      sing[nsing++] = a + 1.0 / al;
    } else if (f == 8) {
      const double xl = -2.0 + 4.0 * p[0], xr = -2.0 + 4.0 * p[1];
      const int shift = p[2] < 0.5 ? 0 : -2 + min((int)(5.0 * p[3]), 4);
      const double xj = xi + (0.5 + shift) * dx;
      for (int j = 0; j < 6; ++j) F[j] = x[j] <= xj ? xl : xr;
      sing[nsing++] = xj;
    } else {
      const double a1 = 2.0 * p[0], x0 = 2.0 * p[1], Nf = (0.125 + 0.375 * p[2]) * N;
      for (int j = 0; j < 6; ++j) F[j] = a1 * sin((Nf * pi) * (x[j] - x0));
    }
    unsigned eta = 0;
    if (f >= 4 && f <= 8) {
      for (int k = 0; k < 4; ++k) {
        const double lo = xi + kSpan[k][0] * dx, hi = xi + kSpan[k][1] * dx;
        bool hit = false;
        if (f == 4) {  // is some multiple m P strictly inside?
          // P >= 2 dx and the span is at most 3 dx: two or three multiples to test
          double m = floor(lo / period);
          for (int it = 0; it < 8 && m * period < hi; ++it, m = m + 1.0) hit = hit || m * period > lo;
        } else {
          for (int s = 0; s < nsing; ++s) hit = hit || (lo < sing[s] && sing[s] < hi);
        }
        if (hit) eta |= 1u << k;
      }
    } else if (f == 9) {
      eta = teno_labels(T, F);
    }
    const double sg = q[8] < 0.5 ? -1.0 : 1.0;
    double m = 1.0;
    for (int j = 0; j < 6; ++j) {
      F[j] = sg * F[j];
      m = fmax(m, fabs(F[j]));
    }
    for (int j = 0; j < 6; ++j) X[r * 6 + j] = F[j] / m;
    labels[r] = (uint8_t)eta;
    if (family) family[r] = (uint8_t)f;
  }
}

}  // namespace

cudaError_t launch_datagen(const double* u, long long n, double* X, uint8_t* labels, uint8_t* family,
                           int* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 64);
  datagen_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(u, n, X, labels, family, status, teno_tables());
  return cudaGetLastError();
}

}  // namespace neno6
