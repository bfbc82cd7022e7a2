// neno6_step_noalloc: the SSP-RK3 step of neno6_step for callers that must
// not allocate device memory.  Its scratch (two stage states, the CFL maxima,
// dt, t and a status word) is one file-scope static device array, created
// when the library's module is loaded on a device and kept until the process
// exits.  The kernels are the ones neno6_step launches.
#include <cuda.h>

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
// Per device: the array's device address and the id of the context it was
// taken in.  A device reset (or a release of the primary context) loads the
// module again, possibly elsewhere; a changed context id makes the next call
// look the address up again instead of writing through a stale pointer.
struct ScratchSlot {
  unsigned long long ctx_id;
  double* addr;
};
ScratchSlot g_slot[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Driver calls reached through the runtime's entry-point query (the library
// links no driver library): the current context and its process-unique id.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    resolved = true;
  }
  CUcontext ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the static array on the current device.  The name
// g_noalloc_scratch is a host-side stand-in in host code, never a device
// address, so it is looked up with that device current: once per device and
// context (every call when the context id cannot be read).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  unsigned long long id = 0;
  if (g_slot[dev].addr && current_context_id(&id) && id == g_slot[dev].ctx_id) {
    *out = g_slot[dev].addr;
    return cudaSuccess;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  // the lookup made the device's primary context current if it was not
  const bool have_id = current_context_id(&id);
  g_slot[dev].ctx_id = have_id ? id : 0ull;
  g_slot[dev].addr = have_id ? static_cast<double*>(p) : nullptr;
  *out = static_cast<double*>(p);
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
  if (c.mask_mode < NENO6_MASK_MLP || c.mask_mode > NENO6_MASK_TENO6) return NENO6_ERR_ARG;
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
  scheme_tables(c.linear_weights, d, p.a.cand, p.a.wtab);
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
  if (c.mask_mode == kMaskTeno) teno_tables(p.a.teno);
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
