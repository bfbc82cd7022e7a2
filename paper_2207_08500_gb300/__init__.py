"""Python binding of libneno6.so (the NENO6 Euler right-hand side on GB300).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory and the current stream; the
library itself sees plain device pointers (include/neno6.h).  There is no CPU
fallback: importing works without a GPU, but constructing a solver requires
the built library and a CUDA device, and fails loudly otherwise.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libneno6.so")
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(_HERE), "weights", "neno6_mlp_6x64x32x16x8x4.bin")

OK = 0
ERRORS = {-1: "ARG", -2: "SHAPE", -3: "ALIGN", -4: "WEIGHTS", -5: "CUDA", -6: "NONPHYSICAL",
          -7: "TIMEOUT", -8: "UNSUPPORTED"}
PRECISION = {"fp64": 0, "bf16": 1, "fp16": 2}
BC = {"periodic": 0, "transmissive": 1}
LINEAR_WEIGHTS = {"paper": 0, "sixth": 1}
DATAGEN_DRAWS = 9  # uniform draws per training sample (neno6_datagen)
MASK_MODE = {"mlp": 0, "smooth": 1, "rough": 2, "teno6": 3}
LAW = {"advection": 0, "burgers": 1}
# logit band re-evaluated in FP32 by the mixed-precision path
DEFAULT_GUARD_TAU = {"fp64": 0.0, "bf16": 1.0, "fp16": 0.5}

# Public C symbols declared in include/neno6.h (checked by the tests).
EXPORTS = ("neno6_create", "neno6_destroy", "neno6_mask_bytes", "neno6_rhs", "neno6_step",
           "neno6_step_host", "neno6_classify", "neno6_status", "neno6_last_error", "neno6_step_noalloc",
           "neno6_rhs_vjp", "neno6_mlp_bwd", "neno6_guard_count", "neno6_mlp_train",
           "neno6_scalar_rhs", "neno6_scalar_solve", "neno6_pipe_peak", "neno6_datagen")


class Neno6Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("gamma", ctypes.c_double),
                ("bc", ctypes.c_int * 2), ("precision", ctypes.c_int),
                ("linear_weights", ctypes.c_int), ("mask_mode", ctypes.c_int),
                ("guard_tau", ctypes.c_double)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libneno6.so and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libneno6.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2207_08500_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, i64, u8p, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    lib.neno6_create.argtypes = [ctypes.POINTER(_Config), ctypes.c_char_p, ctypes.POINTER(vp)]
    lib.neno6_destroy.argtypes = [vp]
    lib.neno6_mask_bytes.argtypes = [vp]
    lib.neno6_mask_bytes.restype = i64
    lib.neno6_rhs.argtypes = [vp, dp, dp, u8p, u8p, vp]
    lib.neno6_step.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, dp, dp, vp]
    lib.neno6_step_host.argtypes = [vp, dp, dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.neno6_classify.argtypes = [vp, dp, i64, u8p, dp, vp]
    lib.neno6_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp]
    lib.neno6_last_error.argtypes = [vp]
    lib.neno6_last_error.restype = ctypes.c_char_p
    lib.neno6_rhs_vjp.argtypes = [vp, dp, dp, u8p, dp, vp]
    lib.neno6_mlp_bwd.argtypes = [vp, dp, u8p, i64, vp, vp, vp]
    lib.neno6_mlp_train.argtypes = [vp, dp, u8p, i64, vp, i64, ctypes.c_int, vp, vp, vp, i64,
                                    ctypes.c_double, vp, vp]
    lib.neno6_scalar_rhs.argtypes = [vp, ctypes.c_int, dp, dp, u8p, vp]
    lib.neno6_scalar_solve.argtypes = [vp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int64), vp]
    lib.neno6_pipe_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
    lib.neno6_datagen.argtypes = [vp, dp, i64, dp, u8p, u8p, vp]
    lib.neno6_guard_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, vp]
    lib.neno6_step_noalloc.argtypes = [ctypes.POINTER(_Config), dp, i64, dp, ctypes.c_double,
                                       ctypes.c_double, dp, dp, vp, vp]
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Neno6:
    """A grid + scheme configuration bound to the current CUDA device.

    States are float64 CUDA tensors [nv, ny, nx] (nv = 3 in 1D, 4 in 2D) of
    conserved variables (rho, rho u, [rho v], E).
    """

    def __init__(self, ndim=2, nx=64, ny=64, dx=None, dy=None, gamma=1.4,
                 bc=("periodic", "periodic"), precision="fp64", linear_weights="paper",
                 mask_mode="mlp", weights=DEFAULT_WEIGHTS, guard_tau=None):
        if not torch.cuda.is_available():
            raise RuntimeError("NENO6 needs a CUDA device; there is no CPU fallback")
        lib = load_library()
        if ndim == 1:
            ny = 1
        self.ndim, self.nx, self.ny = ndim, nx, ny
        self.nv = 4 if ndim == 2 else 3
        c = _Config()
        c.ndim, c.nx, c.ny = ndim, nx, ny
        c.dx = 1.0 / nx if dx is None else dx
        c.dy = 1.0 / ny if dy is None else dy
        c.gamma = gamma
        c.bc[0], c.bc[1] = BC[bc[0]], BC[bc[1]]
        c.precision = PRECISION[precision]
        c.linear_weights = LINEAR_WEIGHTS[linear_weights]
        c.mask_mode = MASK_MODE[mask_mode]
        if guard_tau is None:
            guard_tau = DEFAULT_GUARD_TAU.get(precision, 0.0)
        c.guard_tau = float(guard_tau)
        self.config = c
        self.weights = weights
        h = ctypes.c_void_p()
        torch.cuda.init()
        rc = lib.neno6_create(ctypes.byref(c), os.fsencode(weights), ctypes.byref(h))
        if rc != OK:
            raise Neno6Error(rc, lib.neno6_last_error(None).decode())
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.neno6_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise Neno6Error(rc, self._lib.neno6_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.nv, self.ny, self.nx)

    @property
    def mask_bytes(self):
        return int(self._lib.neno6_mask_bytes(self._h))

    def _state(self, U, name="U"):
        if not (U.is_cuda and U.dtype == torch.float64 and U.is_contiguous()
                and tuple(U.shape) == self.shape):
            raise ValueError("%s must be a contiguous float64 CUDA tensor of shape %s"
                             % (name, self.shape))
        return U

    def rhs(self, U, mask_in=None, want_mask=False, out=None):
        """dU/dt = L(U); optionally with a frozen mask (mask_in) and/or the
        classifier mask of this evaluation (want_mask)."""
        U = self._state(U)
        out = torch.empty_like(U) if out is None else self._state(out, "out")
        mask = None
        if want_mask:
            mask = torch.empty(self.mask_bytes, dtype=torch.uint8, device=U.device)
        if mask_in is not None:
            assert mask_in.dtype == torch.uint8 and mask_in.numel() == self.mask_bytes
            mask_in = mask_in.contiguous()
        self._check(self._lib.neno6_rhs(self._h, _ptr(U), _ptr(out), _ptr(mask_in), _ptr(mask),
                                        _stream()))
        return (out, mask) if want_mask else out

    def step(self, U, cfl, t_end=0.0, t=None, dt=None):
        """One SSP-RK3 step of U in place.  t / dt: optional float64 CUDA
        scalars (time, advanced on the device; dt of the step)."""
        U = self._state(U)
        self._check(self._lib.neno6_step(self._h, _ptr(U), float(cfl), float(t_end), _ptr(t),
                                         _ptr(dt), _stream()))
        return U

    def step_host(self, U_host, cfl, t_end=0.0, t=None, out=None):
        """One SSP-RK3 step of a state in host memory (float64 CPU tensor
        [nv, ny, nx], pinned for asynchronous copies): the library copies it
        to the device, steps it and copies the result to `out` (default: a
        new CPU tensor; may be U_host).  t: optional float time, returned
        advanced by dt.  Returns (out, t)."""
        assert not U_host.is_cuda and U_host.dtype == torch.float64
        if not (U_host.is_contiguous() and tuple(U_host.shape) == self.shape):
            raise ValueError("U_host must be a contiguous float64 CPU tensor of shape %s" % (self.shape,))
        if out is None:
            out = torch.empty_like(U_host)
        assert not out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
        assert tuple(out.shape) == self.shape
        tc = None if t is None else ctypes.c_double(float(t))
        self._check(self._lib.neno6_step_host(self._h, _ptr(U_host), _ptr(out), float(cfl),
                                              float(t_end), None if tc is None else ctypes.byref(tc),
                                              _stream()))
        return out, (None if tc is None else tc.value)

    def classify(self, X, want_logits=False):
        """Classifier bits (and logits) of raw stencils X [n, 6] float64."""
        assert X.is_cuda and X.dtype == torch.float64 and X.shape[-1] == 6
        X = X.contiguous()
        n = X.shape[0]
        eta = torch.empty(n, dtype=torch.uint8, device=X.device)
        logits = torch.empty((n, 4), dtype=torch.float64, device=X.device) if want_logits else None
        self._check(self._lib.neno6_classify(self._h, _ptr(X), n, _ptr(eta), _ptr(logits),
                                             _stream()))
        return (eta, logits) if want_logits else eta

    def rhs_vjp(self, U, lam, mask=None, out=None):
        """J^T lam of the right-hand side at U with the classifier mask frozen
        (recomputed from U by the FP64 classifier when mask is None)."""
        U = self._state(U)
        lam = self._state(lam.contiguous(), "lam")
        out = torch.empty_like(U) if out is None else self._state(out, "out")
        if mask is not None:
            assert mask.dtype == torch.uint8 and mask.numel() == self.mask_bytes
            mask = mask.contiguous()
        self._check(self._lib.neno6_rhs_vjp(self._h, _ptr(U), _ptr(lam), _ptr(mask), _ptr(out),
                                            _stream()))
        return out

    def mlp_bwd(self, X, labels):
        """(grad [3228] float32, loss float32 tensor) of the mean BCE of the
        classifier on raw stencils X [n, 6] float64 and label bits [n] uint8."""
        assert X.is_cuda and X.dtype == torch.float64 and X.shape[-1] == 6
        assert labels.is_cuda and labels.dtype == torch.uint8 and labels.numel() == X.shape[0]
        X, labels = X.contiguous(), labels.contiguous()
        grad = torch.empty(3228, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        self._check(self._lib.neno6_mlp_bwd(self._h, _ptr(X), _ptr(labels), X.shape[0], _ptr(grad),
                                            _ptr(loss), _stream()))
        return grad, loss

    def _scalar(self, u, name="u"):
        if not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous() and u.numel() == self.nx
                and u.dim() == 1):
            raise ValueError("%s must be a contiguous float64 CUDA vector of length %d" % (name, self.nx))
        return u

    def scalar_rhs(self, law, u, want_mask=False, out=None):
        """du/dt of the scalar law `law` ("advection" or "burgers") on this
        1D FP64 grid (neno6_scalar_rhs); optionally the face masks [nx+1]."""
        u = self._scalar(u)
        out = torch.empty_like(u) if out is None else self._scalar(out, "out")
        mask = torch.empty(self.nx + 1, dtype=torch.uint8, device=u.device) if want_mask else None
        self._check(self._lib.neno6_scalar_rhs(self._h, LAW[law], _ptr(u), _ptr(out), _ptr(mask),
                                               _stream()))
        return (out, mask) if want_mask else out

    def scalar_solve(self, law, u, cfl, t_end):
        """Advance u in place to t_end at the fixed step cfl dx / max|f'(u0)|
        (neno6_scalar_solve); returns the number of steps."""
        u = self._scalar(u)
        ns = ctypes.c_int64(0)
        self._check(self._lib.neno6_scalar_solve(self._h, LAW[law], _ptr(u), float(cfl), float(t_end),
                                                 ctypes.byref(ns), _stream()))
        return int(ns.value)

    def mlp_train(self, X, labels, perm, params, adam_m, adam_v, adam_t0, lr, batch=175):
        """Mini-batch Adam steps on the classifier loss (neno6_mlp_train):
        batches of `batch` samples in the order of perm (int32 CUDA tensor of
        sample indices).  params / adam_m / adam_v: float32 CUDA tensors
        [3228], updated in place.  Returns the float64 CUDA scalar holding the
        sum over the steps of each batch's mean loss."""
        assert X.is_cuda and X.dtype == torch.float64 and X.shape[-1] == 6
        assert labels.is_cuda and labels.dtype == torch.uint8 and labels.numel() == X.shape[0]
        assert perm.is_cuda and perm.dtype == torch.int32
        for t in (params, adam_m, adam_v):
            assert t.is_cuda and t.dtype == torch.float32 and t.numel() == 3228 and t.is_contiguous()
        X, labels, perm = X.contiguous(), labels.contiguous(), perm.contiguous()
        loss_sum = torch.zeros(1, dtype=torch.float64, device=X.device)
        self._check(self._lib.neno6_mlp_train(self._h, _ptr(X), _ptr(labels), X.shape[0], _ptr(perm),
                                              perm.numel(), int(batch), _ptr(params), _ptr(adam_m),
                                              _ptr(adam_v), int(adam_t0), float(lr), _ptr(loss_sum),
                                              _stream()))
        return loss_sum

    def datagen(self, u):
        """Training samples of Table 9 from uniform draws u (float64 CUDA
        tensor [n, 9], values in [0, 1)): returns (X [n, 6] float64,
        labels [n] uint8, family [n] uint8), all on the device."""
        assert u.is_cuda and u.dtype == torch.float64 and u.dim() == 2 and u.shape[1] == DATAGEN_DRAWS
        u = u.contiguous()
        n = u.shape[0]
        X = torch.empty((n, 6), dtype=torch.float64, device=u.device)
        labels = torch.empty(n, dtype=torch.uint8, device=u.device)
        fam = torch.empty(n, dtype=torch.uint8, device=u.device)
        self._check(self._lib.neno6_datagen(self._h, _ptr(u), n, _ptr(X), _ptr(labels), _ptr(fam),
                                            _stream()))
        return X, labels, fam

    def guard_count(self, reset=False):
        """Synchronise the current stream and return how many classifier rows
        the mixed-precision path re-evaluated in FP32 (guard band) since the
        last reset."""
        v = ctypes.c_uint64(0)
        self._check(self._lib.neno6_guard_count(self._h, ctypes.byref(v), int(bool(reset)),
                                                _stream()))
        return int(v.value)

    def status(self):
        """Synchronise the current stream and return (and clear) the device
        status bits (1: non-physical cell, 2: non-physical Roe state)."""
        v = ctypes.c_int(0)
        rc = self._lib.neno6_status(self._h, ctypes.byref(v), _stream())
        if rc not in (OK, -6):
            self._check(rc)
        return v.value


def pipe_peak(which="fp64"):
    """Measured FMA rate of the current GPU in FLOP/s (neno6_pipe_peak):
    "fp64" (DFMA) or "fp32" (FFMA)."""
    lib = load_library()
    v = ctypes.c_double(0.0)
    rc = lib.neno6_pipe_peak({"fp64": 0, "fp32": 1}[which], ctypes.byref(v), _stream())
    if rc != OK:
        raise Neno6Error(rc, "pipe_peak")
    return v.value


class RHS(torch.autograd.Function):
    """dU/dt = L(U) as a differentiable function: the forward pass is
    neno6_rhs (keeping its classifier mask), the backward pass the frozen-mask
    adjoint neno6_rhs_vjp."""

    @staticmethod
    def forward(ctx, U, solver):
        dUdt, mask = solver.rhs(U.contiguous(), want_mask=True)
        ctx.solver = solver
        ctx.save_for_backward(U, mask)
        return dUdt

    @staticmethod
    def backward(ctx, grad_out):
        U, mask = ctx.saved_tensors
        return ctx.solver.rhs_vjp(U.contiguous(), grad_out.contiguous(), mask=mask), None


def rhs(U, solver):
    """Differentiable NENO6 right-hand side (see RHS)."""
    return RHS.apply(U, solver)
