// C ABI of the NENO6 library (declared in include/neno6.h): handle life
// cycle, weights-file loading, argument checks and kernel launches.  Nothing
// here throws across the ABI; errors are returned as NENO6_ERR_* codes with a
// message kept on the handle.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/neno6.h"
#include "internal.h"

using namespace neno6;

struct neno6_handle {
  neno6_config cfg;
  int nv = 0;
  int device = 0;
  bool narrow = false;        // the 6-32-32-32-4 network (neno6_classify only)
  NetF64 net;                 // host copy of the classifier parameters
  double d[4];                // linear weights
  double cand[4][4];          // candidate coefficients
  double wtab[16][4];         // renormalised weights per mask pattern
  int* d_status = nullptr;    // device status word
  unsigned long long* d_smax = nullptr;  // [2] CFL maxima
  double* d_dt = nullptr;     // dt of the current step
  double* d_t = nullptr;      // internal time (neno6_step with t_dev == NULL)
  double* d_stage = nullptr;  // two RK3 stage states (lazily allocated)
  double* d_host_state = nullptr;  // device copy of neno6_step_host's state (lazily)
  uint8_t* d_net_image = nullptr;  // tensor-core classifier image (mixed precision)
  uint8_t* d_bwd_image = nullptr;  // its backward image (tensor-core gradient)
  float* d_guard_w = nullptr;      // FP32 transposed parameters (guard band)
  double* d_faces = nullptr;       // x- and y-face fluxes (mixed precision, lazily)
  uint8_t* d_mask = nullptr;       // classifier mask of the adjoint's forward pass (lazily)
  double* d_vjp_rhs = nullptr;     // dU/dt of that forward pass (lazily)
  double* d_vjp_contrib = nullptr; // per-face adjoint contributions (lazily)
  float* d_params32 = nullptr;     // FP32 parameters, weights-file order
  void* d_bwd_scratch = nullptr;   // per-CTA partial gradients (lazily)
  unsigned long long* d_guard_count = nullptr;
  cudaStream_t copy_stream = nullptr;  // neno6_step_host: band copies in and out (lazily)
  cudaEvent_t band_in[9] = {};         // band copied in; [8]: the step's stream reached the call
  cudaEvent_t band_done[9] = {};       // band of the last stage done; [8]: all copied out
  FacesMixedArgs faces_args;
  size_t state_elems = 0;
  RhsParamsF64 rhs_params;        // launch parameter blocks (copied at launch)
  ClassifyParamsF64 cls_params;
  ScalarParams scalar_params;
  std::string err;
};

namespace neno6 {

namespace {

// Exact rational arithmetic for the TENO6-opt indicator matrices (small
// numerators and denominators: the six-point matrix's largest denominator
// is 120960), reduced after every operation.
struct Rat {
  __int128 n, d;
};
__int128 gcd128(__int128 a, __int128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    const __int128 r = a % b;
    a = b;
    b = r;
  }
  return a;
}
Rat rat(__int128 n, __int128 d) {
  if (d < 0) {
    n = -n;
    d = -d;
  }
  const __int128 g = gcd128(n, d);
  if (g > 1) {
    n /= g;
    d /= g;
  }
  return Rat{n, d};
}
Rat operator+(Rat a, Rat b) { return rat(a.n * b.d + b.n * a.d, a.d * b.d); }
Rat operator-(Rat a, Rat b) { return rat(a.n * b.d - b.n * a.d, a.d * b.d); }
Rat operator*(Rat a, Rat b) { return rat(a.n * b.n, a.d * b.d); }
Rat operator/(Rat a, Rat b) { return rat(a.n * b.d, a.d * b.n); }
// Correctly rounded binary64 value: numerator and denominator are exact
// doubles (below 2^53), and IEEE division rounds their quotient once.
double to_double(Rat a) {
  const __int128 lim = (__int128)1 << 53;
  if (a.n >= lim || -a.n >= lim || a.d >= lim) return std::nan("");
  return (double)(long long)a.n / (double)(long long)a.d;
}

// B with beta = f^T B f for the cells at offsets o[0..r-1] (unit spacing,
// the central cell at 0): the polynomial p of degree r-1 whose cell averages
// are f has coefficients a = A^-1 f, A_jl = integral of x^l over cell o_j;
// the Jiang-Shu indicator sum_{l=1}^{r-1} integral over [-1/2, 1/2] of
// (d^l p / dx^l)^2 is then a^T M a.
void beta_rational(const int* o, int r, double* out) {
  Rat A[6][12];
  for (int j = 0; j < r; ++j) {
    const Rat hi = rat(2 * o[j] + 1, 2), lo = rat(2 * o[j] - 1, 2);
    Rat ph = hi, pl = lo;  // hi^(l+1), lo^(l+1)
    for (int l = 0; l < r; ++l) {
      A[j][l] = (ph - pl) / rat(l + 1, 1);
      ph = ph * hi;
      pl = pl * lo;
    }
    for (int l = 0; l < r; ++l) A[j][r + l] = rat(j == l ? 1 : 0, 1);
  }
  for (int c = 0; c < r; ++c) {  // Gauss-Jordan: [A | I] -> [I | A^-1]
    int piv = c;
    while (A[piv][c].n == 0) ++piv;
    if (piv != c)
      for (int l = 0; l < 2 * r; ++l) std::swap(A[c][l], A[piv][l]);
    const Rat d = A[c][c];
    for (int l = 0; l < 2 * r; ++l) A[c][l] = A[c][l] / d;
    for (int j = 0; j < r; ++j) {
      if (j == c || A[j][c].n == 0) continue;
      const Rat f = A[j][c];
      for (int l = 0; l < 2 * r; ++l) A[j][l] = A[j][l] - f * A[c][l];
    }
  }
  // M_pq = sum_l p!/(p-l)! q!/(q-l)! integral of x^(p+q-2l) over [-1/2, 1/2]
  Rat M[6][6];
  for (int p = 0; p < r; ++p)
    for (int q = 0; q < r; ++q) {
      M[p][q] = rat(0, 1);
      for (int l = 1; l <= p && l <= q; ++l) {
        const int m = p + q - 2 * l;
        if (m % 2) continue;
        __int128 fp = 1, fq = 1;
        for (int t = 0; t < l; ++t) {
          fp *= p - t;
          fq *= q - t;
        }
        M[p][q] = M[p][q] + rat(fp * fq, ((__int128)1 << m) * (m + 1));
      }
    }
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      Rat b = rat(0, 1);
      for (int p = 0; p < r; ++p)
        for (int q = 0; q < r; ++q) b = b + A[p][r + i] * M[p][q] * A[q][r + j];
      out[i * r + j] = to_double(b);
    }
}

}  // namespace

void teno_tables(double out[kTenoTable]) {
  static const std::vector<double> t = [] {
    std::vector<double> x(kTenoTable);
    const int s0[3] = {-1, 0, 1}, s1[3] = {0, 1, 2}, s2[3] = {-2, -1, 0}, s3[4] = {0, 1, 2, 3};
    const int full[6] = {-2, -1, 0, 1, 2, 3};
    beta_rational(s0, 3, &x[0]);
    beta_rational(s1, 3, &x[9]);
    beta_rational(s2, 3, &x[18]);
    beta_rational(s3, 4, &x[27]);
    beta_rational(full, 6, &x[43]);
    return x;
  }();
  std::memcpy(out, t.data(), sizeof(double) * kTenoTable);
}

void scheme_tables(int linear_weights, double d[4], double cand[4][4], double wtab[16][4]) {
  if (linear_weights == NENO6_W_SIXTH) {
    d[0] = 9.0 / 20.0;
    d[1] = 3.0 / 10.0;
    d[2] = 1.0 / 20.0;
    d[3] = 1.0 / 5.0;
  } else {  // Sec. 2.2 / Sec. 4 (TENO6-opt optimal weights)
    d[0] = 0.4294317718960898;
    d[1] = 0.1727270875843552;
    d[2] = 0.0855682281039113;
    d[3] = 0.312272912415645;
  }
  // Reconstruction of h(x_{i+1/2}) from point values acting as cell averages
  // (Eqs. (definitionEq), (approximatepolynomial)) on S0 = {i-1,i,i+1},
  // S1 = {i,i+1,i+2}, S2 = {i-2,i-1,i}, S3 = {i,i+1,i+2,i+3}.
  const double c[4][4] = {{-1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0},
                          {1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0, 0.0},
                          {1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0, 0.0},
                          {1.0 / 4.0, 13.0 / 12.0, -5.0 / 12.0, 1.0 / 12.0}};
  std::memcpy(cand, c, sizeof c);
  // Eq. (TENOweight_renormalize): w_k = d_k delta_k / sum_k d_k delta_k,
  // the sum taken over the kept stencils in k order.
  for (int eta = 0; eta < 16; ++eta) {
    double D = 0.0;
    for (int k = 0; k < 4; ++k)
      if (!((eta >> k) & 1)) D = D + d[k];
    for (int k = 0; k < 4; ++k) wtab[eta][k] = (!((eta >> k) & 1) && D != 0.0) ? d[k] / D : 0.0;
  }
}

}  // namespace neno6

namespace {

std::string g_create_error;

int fail(neno6_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(neno6_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, NENO6_ERR_CUDA, m);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// FNV-1a 64-bit over the payload (weights-file integrity check).
uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 0xCBF29CE484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

int32_t rd_i32(const unsigned char* p) {
  uint32_t v = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
  int32_t r;
  std::memcpy(&r, &v, 4);
  return r;
}

uint64_t rd_u64(const unsigned char* p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

double rd_f64(const unsigned char* p) {
  uint64_t v = rd_u64(p);
  double d;
  std::memcpy(&d, &v, 8);
  return d;
}

int load_weights(const char* path, NetF64& net, bool& narrow, std::string& msg) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    msg = std::string("cannot open weights file ") + path;
    return NENO6_ERR_WEIGHTS;
  }
  std::vector<unsigned char> buf;
  unsigned char tmp[65536];
  size_t n;
  while ((n = std::fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
  std::fclose(f);
  if (buf.size() < 16 || std::memcmp(buf.data(), "NENO6W01", 8) != 0) {
    msg = "weights file: bad magic";
    return NENO6_ERR_WEIGHTS;
  }
  // the paper's 6-64-32-16-8-4 network, or the width study's 6-32-32-32-4
  const int32_t nl = rd_i32(&buf[8]);
  narrow = nl == 4;
  const int* widths = narrow ? kNarrowWidths : kNetWidths;
  const size_t nparams = narrow ? kNarrowParams : kNetParams;
  const size_t expect = 8 + 4 + 4 * (size_t)(nl + 1) + 8 * nparams + 8;
  bool ok = (nl == 5 || nl == 4) && buf.size() == expect;
  for (int l = 0; ok && l <= nl; ++l) ok = rd_i32(&buf[12 + 4 * l]) == widths[l];
  if (!ok) {
    msg = "weights file: widths must be 6-64-32-16-8-4 (or 6-32-32-32-4 for neno6_classify)";
    return NENO6_ERR_WEIGHTS;
  }
  const size_t payload = buf.size() - 16;
  if (fnv1a64(&buf[8], payload) != rd_u64(&buf[buf.size() - 8])) {
    msg = "weights file: checksum mismatch";
    return NENO6_ERR_WEIGHTS;
  }
  const unsigned char* p = &buf[12 + 4 * (nl + 1)];
  for (size_t i = 0; i < (size_t)kNetParams; ++i) net.p[i] = i < nparams ? rd_f64(p + 8 * i) : 0.0;
  return NENO6_OK;
}

void fill_tables(neno6_handle* h) { scheme_tables(h->cfg.linear_weights, h->d, h->cand, h->wtab); }

void fill_rhs_args(const neno6_handle* h, RhsArgs& a) {
  std::memset(&a, 0, sizeof a);
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.bcx = h->cfg.bc[0];
  a.bcy = h->cfg.bc[1];
  a.dx = h->cfg.dx;
  a.dy = h->cfg.dy;
  a.gamma = h->cfg.gamma;
  a.gm1 = h->cfg.gamma - 1.0;
  a.third = 1.0 / 3.0;
  a.two_thirds = 2.0 / 3.0;
  a.mask_mode = h->cfg.mask_mode;
  a.status = h->d_status;
  std::memcpy(a.cand, h->cand, sizeof a.cand);
  std::memcpy(a.wtab, h->wtab, sizeof a.wtab);
  if (a.mask_mode == kMaskTeno) teno_tables(a.teno);
}

size_t face_elems(const neno6_handle* h) {
  const size_t nx = h->cfg.nx, ny = h->cfg.ny, nv = h->nv;
  return nv * ny * (nx + 1) + (h->cfg.ndim == 2 ? nv * (ny + 1) * nx : 0);
}

int ensure_faces(neno6_handle* h) {
  if (h->d_faces) return NENO6_OK;
  cudaError_t e = cudaMalloc(&h->d_faces, face_elems(h) * sizeof(double));
  if (e != cudaSuccess) {
    h->d_faces = nullptr;
    return cuda_fail(h, e, "face-flux buffers");
  }
  return NENO6_OK;
}

int ensure_stage(neno6_handle* h) {
  if (h->d_stage) return NENO6_OK;
  cudaError_t e = cudaMalloc(&h->d_stage, 2 * h->state_elems * sizeof(double));
  if (e != cudaSuccess) {
    h->d_stage = nullptr;
    return cuda_fail(h, e, "step: stage buffers");
  }
  return NENO6_OK;
}

// Face-kernel arguments of a mixed-precision RHS evaluation of U.
void fill_faces_args(neno6_handle* h, const double* U, uint8_t* mask_out) {
  FacesMixedArgs& a = h->faces_args;
  std::memset(&a, 0, sizeof a);
  a.U = U;
  a.Fx = h->d_faces;
  a.Fy = h->d_faces + (size_t)h->nv * h->cfg.ny * (h->cfg.nx + 1);
  a.mask_out = mask_out;
  a.status = h->d_status;
  a.net_image = h->d_net_image;
  a.guard_w = h->d_guard_w;
  a.guard_count = h->d_guard_count;
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.bcx = h->cfg.bc[0];
  a.bcy = h->cfg.bc[1];
  a.mask_mode = h->cfg.mask_mode;
  a.bf16 = h->cfg.precision == NENO6_MIXED_BF16;
  a.guard_tau = (float)h->cfg.guard_tau;
  a.gamma = h->cfg.gamma;
  a.gm1 = h->cfg.gamma - 1.0;
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l) a.cand[k][l] = (float)h->cand[k][l];
  for (int e = 0; e < 16; ++e)
    for (int k = 0; k < 4; ++k) a.wtab[e][k] = (float)h->wtab[e][k];
}

// Difference-kernel arguments for the rows j0 .. j1 - 1.
DiffArgs diff_args(const neno6_handle* h, const double* U, const double* U0, double* out, int stage,
                   double* t_dev, int j0, int j1) {
  DiffArgs d;
  d.Fx = h->faces_args.Fx;
  d.Fy = h->faces_args.Fy;
  d.U = U;
  d.U0 = U0;
  d.out = out;
  d.dt_dev = h->d_dt;
  d.t_dev = t_dev;
  d.nx = h->cfg.nx;
  d.ny = h->cfg.ny;
  d.stage = stage;
  d.bcx = h->cfg.bc[0];
  d.bcy = h->cfg.bc[1];
  d.j0 = j0;
  d.j1 = j1;
  d.inv_dx = 1.0 / h->cfg.dx;
  d.inv_dy = 1.0 / h->cfg.dy;
  d.third = 1.0 / 3.0;
  d.two_thirds = 2.0 / 3.0;
  return d;
}

// One mixed-precision RHS evaluation of U; stage 0 writes dU/dt to out,
// stages 1..3 the RK3 stage state (dt from h->d_dt).
int mixed_rhs(neno6_handle* h, const double* U, const double* U0, double* out, int stage, uint8_t* mask_out,
              double* t_dev, cudaStream_t s) {
  int rc = ensure_faces(h);
  if (rc != NENO6_OK) return rc;
  fill_faces_args(h, U, mask_out);
  cudaError_t e = launch_faces_mixed(h->cfg.ndim, h->faces_args, s, 0, h->cfg.ny);
  if (e != cudaSuccess) return cuda_fail(h, e, "mixed face kernel");
  e = launch_diff_mixed(h->cfg.ndim, diff_args(h, U, U0, out, stage, t_dev, 0, h->cfg.ny), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "mixed difference kernel");
  return NENO6_OK;
}

// Row bands of a host-state step on the mixed path, as boundaries
// b[0] = 0 < b[1] < ... < b[nb] = ny (multiples of 16 but the last); returns
// nb <= 8.  From 1024 rows a 128-row first and last band around six equal
// ones: the copy in before the first face kernel and the copy out after the
// last difference are what the overlap leaves exposed.  From 256 rows eight
// equal bands; below, and in 1D, one band.
int band_bounds(const neno6_handle* h, int b[9]) {
  const int ny = h->cfg.ny;
  int nb = 0;
  b[nb++] = 0;
  if (h->cfg.ndim == 2 && ny >= 1024) {
    constexpr int kEdge = 128;
    const int last0 = (ny - kEdge) / 16 * 16;
    const int mid = ((last0 - kEdge + 5) / 6 + 15) / 16 * 16;
    for (int r = kEdge; r < last0; r += mid) b[nb++] = r;
    b[nb++] = last0;
  } else if (h->cfg.ndim == 2 && ny >= 256) {
    const int rows = ((ny + 7) / 8 + 15) / 16 * 16;
    for (int r = rows; r < ny; r += rows) b[nb++] = r;
  }
  b[nb] = ny;
  return nb;
}

int ensure_copy_stream(neno6_handle* h) {
  if (h->copy_stream) return NENO6_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
  for (int b = 0; b < 9 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&h->band_in[b], cudaEventDisableTiming);
  for (int b = 0; b < 9 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&h->band_done[b], cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host: copy stream");
  return NENO6_OK;
}

// Copy rows r0 .. r1 - 1 of every field between a host state and a device
// state (both [nv][ny][nx]).
cudaError_t copy_rows(const neno6_handle* h, double* dst, const double* src, int r0, int r1, cudaMemcpyKind kind,
                      cudaStream_t s) {
  const size_t plane = (size_t)h->cfg.nx * h->cfg.ny;
  cudaError_t e = cudaSuccess;
  for (int n = 0; n < h->nv && e == cudaSuccess; ++n) {
    const size_t off = n * plane + (size_t)r0 * h->cfg.nx;
    e = cudaMemcpyAsync(dst + off, src + off, (size_t)(r1 - r0) * h->cfg.nx * sizeof(double), kind, s);
  }
  return e;
}

// Mixed-precision SSP-RK3 step of U (CFL reduction, dt, three stages).
// With in_host / out_host (neno6_step_host), U is filled from in_host and
// copied to out_host in row bands on the handle's copy stream, overlapped
// with compute: the first stage's face fluxes (which do not depend on dt)
// and the wave-speed maxima of each band start as soon as the band and the
// rows its stencils read have arrived, only the first stage's difference
// waits for dt;
// the last stage runs band by band (face kernel of band b + 1, then the
// difference of band b, whose top row needs the first y faces of band b + 1),
// each band copied out as it finishes.  The arithmetic of every face and
// cell, and dt (a maximum), are those of the unbanded step.  Stream s waits
// for the copies before this returns.
int mixed_step(neno6_handle* h, double* U, double cfl, double t_end, double* t_dev, double* dt_dev,
               const double* in_host, double* out_host, cudaStream_t s) {
  int rc = ensure_faces(h);
  if (rc == NENO6_OK && (in_host || out_host)) rc = ensure_copy_stream(h);
  if (rc != NENO6_OK) return rc;
  const int ndim = h->cfg.ndim, nx = h->cfg.nx, ny = h->cfg.ny;
  double* S1 = h->d_stage;
  double* S2 = h->d_stage + h->state_elems;
  double* tp = t_dev ? t_dev : h->d_t;
  int bounds[9] = {0, ny};
  const int nb = (in_host || out_host) ? band_bounds(h, bounds) : 1;
  auto r0_of = [&](int b) { return bounds[b]; };
  auto r1_of = [&](int b) { return bounds[b + 1]; };
  cudaError_t e = cudaSuccess;
  // ---- stage 1: bands in, wave-speed maxima, face fluxes
  fill_faces_args(h, U, nullptr);
  if (in_host) {
    // A band's y faces read three rows of each neighbouring band, so the
    // copies run: the last band's final kHalo rows (the periodic wrap of band
    // 0), then each band with the first kHalo rows of the next; band b's
    // wave-speed maxima and face fluxes start as soon as that much is in.
    constexpr int kHalo = 16;
    const int tail0 = nb >= 2 ? ny - kHalo : ny;
    e = cudaEventRecord(h->band_in[8], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->band_in[8], 0);
    if (e == cudaSuccess && tail0 < ny)
      e = copy_rows(h, U, in_host, tail0, ny, cudaMemcpyHostToDevice, h->copy_stream);
    int copied = 0;  // rows [0, copied) are in (and [tail0, ny))
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
      int hi = b + 1 < nb ? r1_of(b) + kHalo : tail0;
      if (hi > tail0) hi = tail0;
      if (hi > copied) {
        e = copy_rows(h, U, in_host, copied, hi, cudaMemcpyHostToDevice, h->copy_stream);
        copied = hi;
      }
      if (e == cudaSuccess) e = cudaEventRecord(h->band_in[b], h->copy_stream);
    }
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
      e = cudaStreamWaitEvent(s, h->band_in[b], 0);
      if (e == cudaSuccess)
        e = launch_cfl_mixed(ndim, U, nx, ny, h->cfg.gamma, h->d_smax, h->d_status, s, r0_of(b), r1_of(b), b == 0);
      if (e == cudaSuccess) e = launch_faces_mixed(ndim, h->faces_args, s, r0_of(b), r1_of(b));
    }
  } else {
    e = launch_cfl_mixed(ndim, U, nx, ny, h->cfg.gamma, h->d_smax, h->d_status, s, 0, ny, true);
    if (e == cudaSuccess) e = launch_faces_mixed(ndim, h->faces_args, s, 0, ny);
  }
  if (e == cudaSuccess) e = launch_dt(h->d_smax, ndim, h->cfg.dx, h->cfg.dy, cfl, t_end, tp, h->d_dt, dt_dev, s);
  if (e == cudaSuccess) e = launch_diff_mixed(ndim, diff_args(h, U, U, S1, 1, tp, 0, ny), s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step: first stage");
  // ---- stage 2
  rc = mixed_rhs(h, S1, U, S2, 2, nullptr, tp, s);
  if (rc != NENO6_OK) return rc;
  // ---- stage 3
  if (!out_host) return mixed_rhs(h, S2, U, U, 3, nullptr, tp, s);
  fill_faces_args(h, S2, nullptr);
  e = launch_faces_mixed(ndim, h->faces_args, s, r0_of(0), r1_of(0));
  for (int b = 0; b < nb && e == cudaSuccess; ++b) {
    if (b + 1 < nb) {
      e = launch_faces_mixed(ndim, h->faces_args, s, r0_of(b + 1), r1_of(b + 1));
      if (e != cudaSuccess) break;
    }
    e = launch_diff_mixed(ndim, diff_args(h, S2, U, U, 3, b == 0 ? tp : nullptr, r0_of(b), r1_of(b)), s);
    if (e == cudaSuccess) e = cudaEventRecord(h->band_done[b], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->band_done[b], 0);
    if (e == cudaSuccess) e = copy_rows(h, out_host, U, r0_of(b), r1_of(b), cudaMemcpyDeviceToHost, h->copy_stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->band_done[8], h->copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->band_done[8], 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host: last stage in bands");
  return NENO6_OK;
}

}  // namespace

extern "C" {

int neno6_create(const neno6_config* cfg, const char* weights_path, neno6_handle** out) {
  if (!cfg || !weights_path || !out) return fail(nullptr, NENO6_ERR_ARG, "null argument");
  *out = nullptr;
  const neno6_config& c = *cfg;
  if (c.ndim != 1 && c.ndim != 2) return fail(nullptr, NENO6_ERR_ARG, "ndim must be 1 or 2");
  if (c.nx < 1 || c.ny < 1 || (c.ndim == 1 && c.ny != 1))
    return fail(nullptr, NENO6_ERR_SHAPE, "need nx >= 1, ny >= 1 (ny == 1 in 1D)");
  if ((long long)c.nx * c.ny > (1ll << 34) || c.nx > (1 << 30) || c.ny > (1 << 30))
    return fail(nullptr, NENO6_ERR_SHAPE, "grid too large");
  if (!(c.dx > 0.0) || (c.ndim == 2 && !(c.dy > 0.0)) || !(c.gamma > 1.0))
    return fail(nullptr, NENO6_ERR_ARG, "need dx, dy > 0 and gamma > 1");
  for (int k = 0; k < 2; ++k)
    if (c.bc[k] != NENO6_BC_PERIODIC && c.bc[k] != NENO6_BC_TRANSMISSIVE)
      return fail(nullptr, NENO6_ERR_ARG, "bad boundary condition");
  if (c.linear_weights != NENO6_W_PAPER_OPT && c.linear_weights != NENO6_W_SIXTH)
    return fail(nullptr, NENO6_ERR_ARG, "bad linear_weights");
  if (c.mask_mode < NENO6_MASK_MLP || c.mask_mode > NENO6_MASK_TENO6)
    return fail(nullptr, NENO6_ERR_ARG, "bad mask_mode");
  if (c.precision != NENO6_FP64 && c.precision != NENO6_MIXED_BF16 && c.precision != NENO6_MIXED_FP16)
    return fail(nullptr, NENO6_ERR_ARG, "bad precision");
  if (c.mask_mode == NENO6_MASK_TENO6 && c.precision != NENO6_FP64)
    return fail(nullptr, NENO6_ERR_UNSUPPORTED, "the TENO6-opt mask mode needs the FP64 path");

  neno6_handle* h = new (std::nothrow) neno6_handle();
  if (!h) return fail(nullptr, NENO6_ERR_ARG, "out of host memory");
  h->cfg = c;
  h->nv = c.ndim == 2 ? 4 : 3;
  std::string msg;
  int rc = load_weights(weights_path, h->net, h->narrow, msg);
  if (rc != NENO6_OK) {
    delete h;
    return fail(nullptr, rc, msg);
  }
  fill_tables(h);
  h->state_elems = (size_t)h->nv * c.nx * c.ny;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_smax, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_dt, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_t, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_t, 0, sizeof(double));
  if (e == cudaSuccess) {
    std::vector<float> p32(kNetParams);
    for (int i = 0; i < kNetParams; ++i) p32[i] = (float)h->net.p[i];
    e = cudaMalloc(&h->d_params32, kNetParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(h->d_params32, p32.data(), kNetParams * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && c.precision != NENO6_FP64) {
    std::vector<uint8_t> img(kNetImageBytes);
    if (h->narrow)
      build_net_image_narrow(h->net, c.precision == NENO6_MIXED_BF16, img.data());
    else
      build_net_image(h->net, c.precision == NENO6_MIXED_BF16, img.data());
    e = cudaMalloc(&h->d_net_image, kNetImageBytes);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_net_image, img.data(), kNetImageBytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h->narrow) {
      std::vector<uint8_t> bimg(kBwdImageBytes);
      build_bwd_image(h->net, c.precision == NENO6_MIXED_BF16, bimg.data());
      e = cudaMalloc(&h->d_bwd_image, kBwdImageBytes);
      if (e == cudaSuccess)
        e = cudaMemcpy(h->d_bwd_image, bimg.data(), kBwdImageBytes, cudaMemcpyHostToDevice);
    }
    std::vector<float> gimg(kNetParams);
    build_guard_image(h->net, gimg.data());
    if (e == cudaSuccess) e = cudaMalloc(&h->d_guard_w, kNetParams * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(h->d_guard_w, gimg.data(), kNetParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_guard_count, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_guard_count, 0, sizeof(unsigned long long));
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    std::string m = std::string("device setup: ") + cudaGetErrorString(e);
    neno6_destroy(h);
    return fail(nullptr, NENO6_ERR_CUDA, m);
  }
  *out = h;
  return NENO6_OK;
}

int neno6_destroy(neno6_handle* h) {
  if (!h) return NENO6_OK;
  cudaDeviceSynchronize();
  cudaFree(h->d_status);
  cudaFree(h->d_smax);
  cudaFree(h->d_dt);
  cudaFree(h->d_t);
  cudaFree(h->d_stage);
  cudaFree(h->d_host_state);
  cudaFree(h->d_net_image);
  cudaFree(h->d_bwd_image);
  cudaFree(h->d_guard_w);
  cudaFree(h->d_faces);
  cudaFree(h->d_guard_count);
  cudaFree(h->d_mask);
  cudaFree(h->d_vjp_rhs);
  cudaFree(h->d_vjp_contrib);
  cudaFree(h->d_params32);
  cudaFree(h->d_bwd_scratch);
  for (cudaEvent_t ev : h->band_in)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : h->band_done)
    if (ev) cudaEventDestroy(ev);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
  return NENO6_OK;
}

int64_t neno6_mask_bytes(const neno6_handle* h) {
  if (!h) return NENO6_ERR_ARG;
  const int64_t nx = h->cfg.nx, ny = h->cfg.ny, nv = h->nv;
  int64_t n = nv * ny * (nx + 1);
  if (h->cfg.ndim == 2) n += nv * (ny + 1) * nx;
  return n;
}

int neno6_rhs(neno6_handle* h, const double* U, double* dUdt, const uint8_t* mask_in,
              uint8_t* mask_out, void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (h->narrow) return fail(h, NENO6_ERR_UNSUPPORTED, "rhs: the 6-32-32-32-4 network serves neno6_classify only");
  if (!U || !dUdt) return fail(h, NENO6_ERR_ARG, "rhs: null state pointer");
  if (h->cfg.precision != NENO6_FP64) {
    if (mask_in) return fail(h, NENO6_ERR_UNSUPPORTED, "rhs: frozen masks need the FP64 path");
    if (!aligned(U, 16) || !aligned(dUdt, 16)) return fail(h, NENO6_ERR_ALIGN, "rhs: U/dUdt must be 16-byte aligned");
    if ((const void*)U == (const void*)dUdt) return fail(h, NENO6_ERR_ARG, "rhs: dUdt must not alias U");
    return mixed_rhs(h, U, U, dUdt, 0, mask_out, h->d_t, (cudaStream_t)stream);
  }
  if (!aligned(U, 16) || !aligned(dUdt, 16)) return fail(h, NENO6_ERR_ALIGN, "rhs: U/dUdt must be 16-byte aligned");
  if ((const void*)U == (const void*)dUdt) return fail(h, NENO6_ERR_ARG, "rhs: dUdt must not alias U");
  RhsParamsF64& p = h->rhs_params;
  fill_rhs_args(h, p.a);
  p.a.U = U;
  p.a.out = dUdt;
  p.a.mask_in = mask_in;
  p.a.mask_out = mask_out;
  if (mask_in) p.a.mask_mode = kMaskGiven;
  p.a.stage = 0;
  p.net = h->net;
  cudaError_t e = launch_rhs_fp64(h->cfg.ndim, p, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "rhs launch");
  return NENO6_OK;
}

int neno6_step(neno6_handle* h, double* U, double cfl, double t_end, double* t_dev, double* dt_dev,
               void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (h->narrow) return fail(h, NENO6_ERR_UNSUPPORTED, "step: the 6-32-32-32-4 network serves neno6_classify only");
  if (!U) return fail(h, NENO6_ERR_ARG, "step: null state pointer");

  if (!aligned(U, 16)) return fail(h, NENO6_ERR_ALIGN, "step: U must be 16-byte aligned");
  if (!(cfl > 0.0) || !(t_end >= 0.0)) return fail(h, NENO6_ERR_ARG, "step: need cfl > 0, t_end >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_stage(h);
  if (rc != NENO6_OK) return rc;
  if (h->cfg.precision != NENO6_FP64) return mixed_step(h, U, cfl, t_end, t_dev, dt_dev, nullptr, nullptr, s);
  double* S1 = h->d_stage;
  double* S2 = h->d_stage + h->state_elems;
  cudaError_t e = launch_cfl_reduce(h->cfg.ndim, U, h->cfg.nx, h->cfg.ny, h->cfg.gamma, h->d_smax, h->d_status, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step: cfl reduction");
  RhsParamsF64& p = h->rhs_params;
  fill_rhs_args(h, p.a);
  p.a.smax = h->d_smax;
  p.a.dt_dev = h->d_dt;
  p.a.t_dev = t_dev ? t_dev : h->d_t;
  p.a.dt_user = dt_dev;
  p.a.cfl = cfl;
  p.a.t_end = t_end;
  p.a.U0 = U;
  p.net = h->net;
  const double* in[3] = {U, S1, S2};
  double* outp[3] = {S1, S2, U};
  for (int st = 1; st <= 3; ++st) {
    p.a.stage = st;
    p.a.U = in[st - 1];
    p.a.out = outp[st - 1];
    e = launch_rhs_fp64(h->cfg.ndim, p, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "step: stage launch");
  }
  return NENO6_OK;
}

int neno6_step_host(neno6_handle* h, const double* U_in, double* U_out, double cfl, double t_end,
                    double* t_io, void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (h->narrow) return fail(h, NENO6_ERR_UNSUPPORTED, "step_host: the 6-32-32-32-4 network serves neno6_classify only");
  if (!U_in || !U_out) return fail(h, NENO6_ERR_ARG, "step_host: null state pointer");
  if (!(cfl > 0.0) || !(t_end >= 0.0)) return fail(h, NENO6_ERR_ARG, "step_host: need cfl > 0, t_end >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = h->state_elems * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (!h->d_host_state) {
    // the state, then the caller's time (kept apart from the internal time)
    e = cudaMalloc(&h->d_host_state, bytes + 2 * sizeof(double));
    if (e != cudaSuccess) {
      h->d_host_state = nullptr;
      return cuda_fail(h, e, "step_host: device state");
    }
  }
  double* t_dev = t_io ? h->d_host_state + h->state_elems : nullptr;
  // the mixed path copies the state in and out in row bands, overlapped with
  // its first and last stages
  const bool banded = h->cfg.precision != NENO6_FP64;
  if (!banded) e = cudaMemcpyAsync(h->d_host_state, U_in, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && t_io) e = cudaMemcpyAsync(t_dev, t_io, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host: copy in");
  int rc = banded ? ensure_stage(h) : NENO6_OK;
  if (rc == NENO6_OK)
    rc = banded ? mixed_step(h, h->d_host_state, cfl, t_end, t_dev, nullptr, U_in, U_out, s)
                : neno6_step(h, h->d_host_state, cfl, t_end, t_dev, nullptr, stream);
  if (rc != NENO6_OK) {
    cudaStreamSynchronize(s);  // the copy in reads U_in: finish it before returning
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    return rc;
  }
  if (!banded) e = cudaMemcpyAsync(U_out, h->d_host_state, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && t_io) e = cudaMemcpyAsync(t_io, t_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host: copy out");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host: synchronise");
  return NENO6_OK;
}

int neno6_datagen(neno6_handle* h, const double* u, int64_t n, double* X, uint8_t* labels, uint8_t* family,
                  void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (n < 0 || n >= (1ll << 40)) return fail(h, NENO6_ERR_SHAPE, "datagen: need 0 <= n < 2^40");
  if (n == 0) return NENO6_OK;
  if (!u || !X || !labels) return fail(h, NENO6_ERR_ARG, "datagen: null pointer");
  if (!aligned(u, 8) || !aligned(X, 8)) return fail(h, NENO6_ERR_ALIGN, "datagen: misaligned");
  cudaError_t e = launch_datagen(u, n, X, labels, family, h->d_status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "datagen launch");
  return NENO6_OK;
}

int neno6_classify(neno6_handle* h, const double* X, int64_t n, uint8_t* eta_out, double* logits,
                   void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (n < 0 || n >= (1ll << 31)) return fail(h, NENO6_ERR_SHAPE, "classify: need 0 <= n < 2^31");
  if (n == 0) return NENO6_OK;
  if (!X || !eta_out) return fail(h, NENO6_ERR_ARG, "classify: null pointer");
  if (!aligned(X, 8) || (logits && !aligned(logits, 8))) return fail(h, NENO6_ERR_ALIGN, "classify: misaligned");
  if (h->cfg.precision != NENO6_FP64) {
    cudaError_t e = launch_classify_mixed(X, n, eta_out, logits, h->d_net_image,
                                          h->cfg.precision == NENO6_MIXED_BF16, h->narrow, h->d_status,
                                          (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "classify launch");
    return NENO6_OK;
  }
  ClassifyParamsF64& p = h->cls_params;
  p.X = X;
  p.eta = eta_out;
  p.logits = logits;
  p.n = n;
  p.net = h->net;
  cudaError_t e = launch_classify_fp64(p, h->narrow, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "classify launch");
  return NENO6_OK;
}

int neno6_rhs_vjp(neno6_handle* h, const double* U, const double* lambda, const uint8_t* mask,
                  double* grad_U, void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (h->narrow) return fail(h, NENO6_ERR_UNSUPPORTED, "rhs_vjp: the 6-32-32-32-4 network serves neno6_classify only");
  if (!U || !lambda || !grad_U) return fail(h, NENO6_ERR_ARG, "rhs_vjp: null pointer");
  if (!aligned(U, 16) || !aligned(lambda, 16) || !aligned(grad_U, 16))
    return fail(h, NENO6_ERR_ALIGN, "rhs_vjp: arrays must be 16-byte aligned");
  if (grad_U == U || grad_U == lambda) return fail(h, NENO6_ERR_ARG, "rhs_vjp: grad_U must not alias an input");
  cudaStream_t s = (cudaStream_t)stream;
  RhsParamsF64& p = h->rhs_params;
  if (!mask) {
    // recompute the classifier mask of U with the FP64 path (bit-identical
    // to the forward FP64 right-hand side)
    cudaError_t e = cudaSuccess;
    if (!h->d_mask) e = cudaMalloc(&h->d_mask, (size_t)neno6_mask_bytes(h));
    if (e == cudaSuccess && !h->d_vjp_rhs) e = cudaMalloc(&h->d_vjp_rhs, h->state_elems * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(h, e, "rhs_vjp: mask buffers");
    fill_rhs_args(h, p.a);
    p.a.U = U;
    p.a.out = h->d_vjp_rhs;
    p.a.mask_out = h->d_mask;
    p.a.stage = 0;
    p.net = h->net;
    e = launch_rhs_fp64(h->cfg.ndim, p, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "rhs_vjp: forward");
    mask = h->d_mask;
  }
  if (!h->d_vjp_contrib) {
    cudaError_t e = cudaMalloc(&h->d_vjp_contrib, vjp_scratch_bytes(h->cfg.ndim, h->cfg.nx, h->cfg.ny));
    if (e != cudaSuccess) {
      h->d_vjp_contrib = nullptr;
      return cuda_fail(h, e, "rhs_vjp: contribution buffer");
    }
  }
  fill_rhs_args(h, p.a);
  p.a.U = U;
  p.a.mask_in = mask;
  cudaError_t e = launch_rhs_vjp(h->cfg.ndim, p.a, lambda, grad_U, h->d_vjp_contrib, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "rhs_vjp launch");
  return NENO6_OK;
}

int neno6_mlp_bwd(neno6_handle* h, const double* X, const uint8_t* labels, int64_t n, float* grad, float* loss,
                  void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (h->narrow) return fail(h, NENO6_ERR_UNSUPPORTED, "mlp_bwd: the 6-32-32-32-4 network serves neno6_classify only");
  if (n < 1 || n >= (1ll << 31)) return fail(h, NENO6_ERR_SHAPE, "mlp_bwd: need 1 <= n < 2^31");
  if (!X || !labels || !grad) return fail(h, NENO6_ERR_ARG, "mlp_bwd: null pointer");
  if (!aligned(X, 8) || !aligned(grad, 4) || (loss && !aligned(loss, 4)))
    return fail(h, NENO6_ERR_ALIGN, "mlp_bwd: misaligned");
  if (!h->d_bwd_scratch) {
    cudaError_t e = cudaMalloc(&h->d_bwd_scratch, mlp_bwd_scratch_bytes(1ll << 30));
    if (e != cudaSuccess) {
      h->d_bwd_scratch = nullptr;
      return cuda_fail(h, e, "mlp_bwd: scratch");
    }
  }
  cudaError_t e =
      h->cfg.precision == NENO6_FP64
          ? launch_mlp_bwd(X, labels, n, h->d_params32, grad, loss, h->d_bwd_scratch, (cudaStream_t)stream)
          : launch_mlp_bwd_tc(X, labels, n, h->d_net_image, h->d_bwd_image, h->cfg.precision == NENO6_MIXED_BF16,
                              grad, loss, h->d_bwd_scratch, h->d_status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mlp_bwd launch");
  return NENO6_OK;
}

namespace {

int scalar_check(neno6_handle* h, int law, const void* u, const char* who) {
  if (!h) return NENO6_ERR_ARG;
  if (h->cfg.ndim != 1 || h->cfg.precision != NENO6_FP64)
    return fail(h, NENO6_ERR_UNSUPPORTED, std::string(who) + ": needs a 1D FP64 handle");
  if (h->narrow)
    return fail(h, NENO6_ERR_UNSUPPORTED, std::string(who) + ": the 6-32-32-32-4 network serves neno6_classify only");
  if (law != NENO6_LAW_ADVECTION && law != NENO6_LAW_BURGERS)
    return fail(h, NENO6_ERR_ARG, std::string(who) + ": unknown law");
  if (!u) return fail(h, NENO6_ERR_ARG, std::string(who) + ": null pointer");
  if (!aligned(u, 8)) return fail(h, NENO6_ERR_ALIGN, std::string(who) + ": misaligned");
  return NENO6_OK;
}

// face fluxes of u into h->d_faces (nx + 1 values)
int scalar_faces(neno6_handle* h, int law, const double* u, uint8_t* mask_out, cudaStream_t s) {
  int rc = ensure_faces(h);
  if (rc != NENO6_OK) return rc;
  ScalarParams& p = h->scalar_params;
  fill_rhs_args(h, p.a);
  p.net = h->net;
  p.law = law;
  p.u = u;
  p.F = h->d_faces;
  p.mask_out = mask_out;
  cudaError_t e = launch_scalar_faces(p, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "scalar face kernel");
  return NENO6_OK;
}

}  // namespace

int neno6_scalar_rhs(neno6_handle* h, int law, const double* u, double* dudt, uint8_t* mask_out, void* stream) {
  int rc = scalar_check(h, law, u, "scalar_rhs");
  if (rc != NENO6_OK) return rc;
  if (!dudt) return fail(h, NENO6_ERR_ARG, "scalar_rhs: null pointer");
  if (!aligned(dudt, 8)) return fail(h, NENO6_ERR_ALIGN, "scalar_rhs: misaligned");
  cudaStream_t s = (cudaStream_t)stream;
  rc = scalar_faces(h, law, u, mask_out, s);
  if (rc != NENO6_OK) return rc;
  cudaError_t e = launch_scalar_diff(h->d_faces, u, u, dudt, h->cfg.nx, h->cfg.dx, 0, 0.0, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "scalar difference kernel");
  return NENO6_OK;
}

int neno6_scalar_solve(neno6_handle* h, int law, double* u, double cfl, double t_end, int64_t* nsteps_out,
                       void* stream) {
  int rc = scalar_check(h, law, u, "scalar_solve");
  if (rc != NENO6_OK) return rc;
  if (!(cfl > 0.0) || !(t_end >= 0.0)) return fail(h, NENO6_ERR_ARG, "scalar_solve: need cfl > 0, t_end >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int n = h->cfg.nx;
  if (!h->d_stage) {
    cudaError_t e = cudaMalloc(&h->d_stage, 2 * h->state_elems * sizeof(double));
    if (e != cudaSuccess) {
      h->d_stage = nullptr;
      return cuda_fail(h, e, "scalar_solve: stage buffers");
    }
  }
  // initial wave speed -> the fixed step (one synchronisation)
  cudaError_t e = launch_scalar_speed(u, n, law, h->d_smax, s);
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, h->d_smax, sizeof bits, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "scalar_solve: wave speed");
  double amax;
  std::memcpy(&amax, &bits, sizeof amax);
  if (!(amax > 0.0)) return fail(h, NENO6_ERR_ARG, "scalar_solve: zero wave speed");
  const double dt = cfl * h->cfg.dx / amax;
  double* u1 = h->d_stage;
  double* u2 = h->d_stage + n;
  double t = 0.0;
  int64_t steps = 0;
  const double* in[3] = {u, u1, u2};
  double* out[3] = {u1, u2, u};
  while (t < t_end) {
    double step = dt;
    if (t + step > t_end) step = t_end - t;
    for (int st = 1; st <= 3; ++st) {
      rc = scalar_faces(h, law, in[st - 1], nullptr, s);
      if (rc != NENO6_OK) return rc;
      e = launch_scalar_diff(h->d_faces, in[st - 1], u, out[st - 1], n, h->cfg.dx, st, step, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "scalar stage kernel");
    }
    t = t + step;
    ++steps;
  }
  if (nsteps_out) *nsteps_out = steps;
  return NENO6_OK;
}

int neno6_mlp_train(neno6_handle* h, const double* X, const uint8_t* labels, int64_t n, const int32_t* perm,
                    int64_t n_perm, int batch, float* params, float* adam_m, float* adam_v, int64_t adam_t0,
                    double lr, double* loss_sum, void* stream) {
  if (!h) return NENO6_ERR_ARG;
  if (h->narrow) return fail(h, NENO6_ERR_UNSUPPORTED, "mlp_train: the 6-32-32-32-4 network serves neno6_classify only");
  if (n < 1 || n >= (1ll << 31) || n_perm < 1 || n_perm >= (1ll << 31))
    return fail(h, NENO6_ERR_SHAPE, "mlp_train: need 1 <= n, n_perm < 2^31");
  if (batch < 1 || batch > kMaxTrainBatch) return fail(h, NENO6_ERR_SHAPE, "mlp_train: need 1 <= batch <= 192");
  if (!X || !labels || !perm || !params || !adam_m || !adam_v) return fail(h, NENO6_ERR_ARG, "mlp_train: null pointer");
  if (adam_t0 < 0 || !(lr >= 0.0)) return fail(h, NENO6_ERR_ARG, "mlp_train: need adam_t0 >= 0, lr >= 0");
  if (!aligned(X, 8) || !aligned(perm, 4) || !aligned(params, 4) || !aligned(adam_m, 4) || !aligned(adam_v, 4) ||
      (loss_sum && !aligned(loss_sum, 8)))
    return fail(h, NENO6_ERR_ALIGN, "mlp_train: misaligned");
  MlpTrainArgs a;
  a.X = X;
  a.y = labels;
  a.n = n;
  a.perm = perm;
  a.n_perm = n_perm;
  a.batch = batch;
  a.params = params;
  a.m = adam_m;
  a.v = adam_v;
  a.t0 = adam_t0;
  a.lr = (float)lr;
  a.loss_sum = loss_sum;
  a.status = h->d_status;
  cudaError_t e = launch_mlp_train(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mlp_train launch");
  return NENO6_OK;
}

int neno6_status(neno6_handle* h, int* device_status, void* stream) {
  if (!h || !device_status) return NENO6_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "status");
  *device_status = v;
  if (v) return fail(h, NENO6_ERR_NONPHYSICAL, "non-physical state seen on the device");
  return NENO6_OK;
}

int neno6_guard_count(neno6_handle* h, uint64_t* count, int reset, void* stream) {
  if (!h || !count) return NENO6_ERR_ARG;
  *count = 0;
  if (!h->d_guard_count) return NENO6_OK;  // FP64 handle: no guard band
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->d_guard_count, sizeof v, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(h->d_guard_count, 0, sizeof v, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "guard count");
  *count = (uint64_t)v;
  return NENO6_OK;
}

const char* neno6_last_error(const neno6_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
