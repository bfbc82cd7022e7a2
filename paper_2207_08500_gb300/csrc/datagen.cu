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
// smoothness indicators from the Jiang-Shu definition (the selection the
// FP64 right-hand side uses in its TENO6-opt mask mode).  Output values are
// normalised by Eq. (normalizainput).
//
// This unit is compiled with -fmad=false and evaluates every expression in
// the order written, so grids, positions and singular points are the exact
// binary64 values of the recipe; the transcendental functions (sin, cos,
// exp, log) are CUDA's and may differ from a host library in the last bit.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fp64_ops.cuh"
#include "internal.h"

namespace neno6 {
namespace {

constexpr int kDraws = 9;
constexpr int kThreads = 256;

// TENO6-opt indicator matrices (exact rationals rounded once), passed by
// value as a kernel parameter.
struct TenoTables {
  double t[kTenoTable];
};

// outermost cell offsets of the candidate sub-stencils S_k
__constant__ int kSpan[4][2] = {{-1, 1}, {0, 2}, {-2, 0}, {0, 3}};

__device__ double ipow(double b, int k) {
  double r = b;
  for (int t = 1; t < k; ++t) r = r * b;
  return r;
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
      eta = f64ops::teno6_eta(T.t, F);
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
  TenoTables T;
  teno_tables(T.t);
  datagen_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(u, n, X, labels, family, status, T);
  return cudaGetLastError();
}

}  // namespace neno6
