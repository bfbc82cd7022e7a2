// neno6_step_noalloc: the SSP-RK3 step of neno6_step for callers that must
// not allocate device memory.  Its scratch (two stage states, the CFL maxima,
// dt, t and a status word) is one file-scope static device array, created
// when the library's module is loaded on a device and kept until the process
// exits.  The kernels are the ones neno6_step launches.
#include <cstring>
#include <mutex>

#include "../../include/neno6.h"
#include "internal.h"

using namespace neno6;

namespace {

// Largest state (nv * nx * ny float64 values) one call may advance.
constexpr size_t kMaxElems = NENO6_NOALLOC_MAX_STATE_ELEMS;
// Layout of the static array, in float64 slots: stage 1, stage 2, then the
// small words (CFL maxima x2, dt, t, status).
constexpr size_t kSmall = 8;
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxElems + kSmall];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the static array on the current device.  The name
// g_noalloc_scratch is a host-side stand-in in host code, never a device
// address, so it is looked up once per device with that device current.
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int neno6_step_noalloc(const neno6_config* cfg, const double* net_params,
                                  int64_t n_params, double* U, double cfl, double t_end,
                                  double* t_dev, double* dt_dev, int* status_dev, void* stream) {
  if (!cfg || !net_params || !U) return NENO6_ERR_ARG;
  const neno6_config& c = *cfg;
  if (c.ndim != 1 && c.ndim != 2) return NENO6_ERR_ARG;
  if (c.precision != NENO6_FP64) return NENO6_ERR_UNSUPPORTED;
  if (c.nx < 1 || c.ny < 1 || (c.ndim == 1 && c.ny != 1)) return NENO6_ERR_SHAPE;
  const int nv = c.ndim == 2 ? 4 : 3;
  const size_t elems = (size_t)nv * (size_t)c.nx * (size_t)c.ny;
  if (elems > kMaxElems) return NENO6_ERR_SHAPE;  // beyond the static scratch
  if (!(c.dx > 0.0) || (c.ndim == 2 && !(c.dy > 0.0)) || !(c.gamma > 1.0)) return NENO6_ERR_ARG;
  for (int k = 0; k < 2; ++k)
    if (c.bc[k] != NENO6_BC_PERIODIC && c.bc[k] != NENO6_BC_TRANSMISSIVE) return NENO6_ERR_ARG;
  if (c.linear_weights != NENO6_W_PAPER_OPT && c.linear_weights != NENO6_W_SIXTH) return NENO6_ERR_ARG;
  if (c.mask_mode < NENO6_MASK_MLP || c.mask_mode > NENO6_MASK_ALL_ROUGH) return NENO6_ERR_ARG;
  if (n_params != kNetParams) return NENO6_ERR_WEIGHTS;
  if (!aligned16(U)) return NENO6_ERR_ALIGN;
  if (!(cfl > 0.0) || !(t_end >= 0.0)) return NENO6_ERR_ARG;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return NENO6_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NENO6_ERR_UNSUPPORTED;
  double* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return NENO6_ERR_CUDA;
  double* S1 = base;
  double* S2 = base + kMaxElems;
  double* small = base + 2 * kMaxElems;
  unsigned long long* smax = reinterpret_cast<unsigned long long*>(small);
  double* dt_s = small + 2;
  double* t_s = small + 3;
  int* status_s = reinterpret_cast<int*>(small + 4);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The array keeps the previous call's contents: clear what starts at zero.
  int* status = status_dev ? status_dev : status_s;
  if (!status_dev) {
    e = cudaMemsetAsync(status_s, 0, sizeof(int), s);
    if (e != cudaSuccess) return NENO6_ERR_CUDA;
  }
  if (!t_dev) {
    e = cudaMemsetAsync(t_s, 0, sizeof(double), s);
    if (e != cudaSuccess) return NENO6_ERR_CUDA;
  }

  // Launch parameters (26 KB; on the stack, no heap allocation).
  RhsParamsF64 p;
  std::memset(&p.a, 0, sizeof p.a);
  std::memcpy(p.net.p, net_params, sizeof p.net.p);
  double d[4];
  if (c.linear_weights == NENO6_W_SIXTH) {
    d[0] = 9.0 / 20.0; d[1] = 3.0 / 10.0; d[2] = 1.0 / 20.0; d[3] = 1.0 / 5.0;
  } else {
    d[0] = 0.4294317718960898; d[1] = 0.1727270875843552;
    d[2] = 0.0855682281039113; d[3] = 0.312272912415645;
  }
  const double cand[4][4] = {{-1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0},
                             {1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0, 0.0},
                             {1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0, 0.0},
                             {1.0 / 4.0, 13.0 / 12.0, -5.0 / 12.0, 1.0 / 12.0}};
  std::memcpy(p.a.cand, cand, sizeof cand);
  for (int eta = 0; eta < 16; ++eta) {
    double D = 0.0;
    for (int k = 0; k < 4; ++k)
      if (!((eta >> k) & 1)) D = D + d[k];
    for (int k = 0; k < 4; ++k) p.a.wtab[eta][k] = (!((eta >> k) & 1) && D != 0.0) ? d[k] / D : 0.0;
  }
  p.a.nx = c.nx;
  p.a.ny = c.ny;
  p.a.bcx = c.bc[0];
  p.a.bcy = c.bc[1];
  p.a.dx = c.dx;
  p.a.dy = c.dy;
  p.a.gamma = c.gamma;
  p.a.gm1 = c.gamma - 1.0;
  p.a.third = 1.0 / 3.0;
  p.a.two_thirds = 2.0 / 3.0;
  p.a.mask_mode = c.mask_mode;
  p.a.status = status;
  p.a.smax = smax;
  p.a.dt_dev = dt_s;
  p.a.t_dev = t_dev ? t_dev : t_s;
  p.a.dt_user = dt_dev;
  p.a.cfl = cfl;
  p.a.t_end = t_end;
  p.a.U0 = U;

  e = launch_cfl_reduce(c.ndim, U, c.nx, c.ny, c.gamma, smax, status, s);
  if (e != cudaSuccess) return NENO6_ERR_CUDA;
  const double* in[3] = {U, S1, S2};
  double* outp[3] = {S1, S2, U};
  for (int st = 1; st <= 3; ++st) {
    p.a.stage = st;
    p.a.U = in[st - 1];
    p.a.out = outp[st - 1];
    e = launch_rhs_fp64(c.ndim, p, s);
    if (e != cudaSuccess) return NENO6_ERR_CUDA;
  }
  return NENO6_OK;
}
