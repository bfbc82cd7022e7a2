"""NENO6 oracle: plain FP64 CPU reference of the NENO6 scheme (arXiv 2207.08500).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this package.  The product library
(paper_2207_08500_gb300) never imports it, and the two share no code.

The arithmetic lives in neno6_oracle.cpp (compiled here with
-ffp-contract=off); this module builds it, loads it with ctypes and marshals
numpy arrays.  Candidate coefficients and linear weights come from
coefficients.py (exact rational derivation), the classifier parameters from
weights.py.

Parity status: everything here is pinned by tests/test_oracle_*.py except
the trained classifier weights themselves (the paper's network is not
available), whose masks are "parity unpinned" against the paper.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import coefficients
from .weights import Net  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "neno6_oracle.cpp")

MASK_MODES = {"mlp": 0, "smooth": 1, "rough": 2, "given": 3, "teno6": 4}
BCS = {"periodic": 0, "transmissive": 1}


def build(force=False):
    """Compile the oracle with the host g++ (no -march, no fast-math, no
    contraction) into oracle/_build/liboracle.so, with OpenMP over the face
    loops where the compiler has it (results are the same either way)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    try:
        subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def set_threads(n=0):
    """Threads of the oracle's face loops for later calls (n >= 1; 0 keeps
    the count); returns the count in force (1 without OpenMP)."""
    return int(_load().oracle_set_threads(int(n)))


class _Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int), ("mask_mode", ctypes.c_int),
        ("n_layers", ctypes.c_int), ("widths", ctypes.c_int * 8),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("gamma", ctypes.c_double),
        ("d", ctypes.c_double * 4), ("cand", (ctypes.c_double * 4) * 4),
        ("net", ctypes.POINTER(ctypes.c_double)),
        ("teno", ctypes.POINTER(ctypes.c_double)),
    ]


_teno_tables = None


def teno_tables():
    """The TENO6-opt smoothness-indicator matrices (S0, S1, S2, S3, full
    stencil; 79 float64 values) of oracle/train/teno6.py, derived exactly from
    the Jiang-Shu definition and rounded once."""
    global _teno_tables
    if _teno_tables is None:
        from .train import teno6
        parts = [teno6.beta_matrix(teno6.STENCILS[k]).ravel() for k in range(4)]
        parts.append(teno6.beta_matrix(teno6.FULL).ravel())
        _teno_tables = np.ascontiguousarray(np.concatenate(parts), dtype=np.float64)
        assert _teno_tables.size == 79
    return _teno_tables


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_rhs.argtypes = [P, dp, dp, u8, u8]
        lib.oracle_rhs_cells.argtypes = [P, dp, ctypes.c_int64, i64p, dp]
        lib.oracle_face_masks.argtypes = [P, dp, ctypes.c_int64, i32p, i32p, i32p, u8]
        lib.oracle_rhs_jvp.argtypes = [P, dp, dp, u8, dp, dp]
        lib.oracle_rhs_jvp_cells.argtypes = [P, dp, dp, u8, ctypes.c_int64, i64p, dp]
        lib.oracle_classify.argtypes = [P, dp, ctypes.c_int64, u8, dp]
        lib.oracle_reconstruct.argtypes = [P, dp, u8]
        lib.oracle_reconstruct.restype = ctypes.c_double
        lib.oracle_roe_eigen.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]
        lib.oracle_dt.argtypes = [P, dp, ctypes.c_double]
        lib.oracle_dt.restype = ctypes.c_double
        lib.oracle_step.argtypes = [P, dp, ctypes.c_double, dp, ctypes.c_double, dp]
        lib.oracle_scalar_solve.argtypes = [P, ctypes.c_int, dp, ctypes.c_double,
                                            ctypes.c_double, i64p]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One grid + scheme configuration.

    U arrays are float64 [nv][ny][nx] (nv = 3 in 1D, 4 in 2D), conserved
    variables (rho, rho u, [rho v], E).
    """

    def __init__(self, ndim=2, nx=16, ny=16, dx=None, dy=None, gamma=1.4,
                 bc=("periodic", "periodic"), net=None, linear_weights="paper",
                 mask_mode="mlp"):
        if ndim == 1:
            ny = 1
        self.ndim, self.nx, self.ny = ndim, nx, ny
        self.nv = 4 if ndim == 2 else 3
        self.net = net if net is not None else Net.random()
        self._packed = _f64(self.net.packed())
        p = _Params()
        p.ndim, p.nx, p.ny = ndim, nx, ny
        p.bc_x, p.bc_y = BCS[bc[0]], BCS[bc[1]]
        p.mask_mode = MASK_MODES[mask_mode]
        w = self.net.widths
        p.n_layers = len(w) - 1
        for i, x in enumerate(w):
            p.widths[i] = x
        p.dx = 1.0 / nx if dx is None else dx
        p.dy = 1.0 / ny if dy is None else dy
        p.gamma = gamma
        self.d = linear_weights if not isinstance(linear_weights, str) \
            else coefficients.linear_weights(linear_weights)
        for k in range(4):
            p.d[k] = self.d[k]
        cand = coefficients.candidate_coefficients()
        for k in range(4):
            for l in range(4):
                p.cand[k][l] = cand[k][l]
        p.net = _ptr(self._packed, ctypes.c_double)
        self._teno = None
        self._p = p
        if mask_mode == "teno6":
            self._attach_teno(p)

    # -- helpers -----------------------------------------------------------
    def _attach_teno(self, p):
        if self._teno is None:
            self._teno = teno_tables()
        p.teno = _ptr(self._teno, ctypes.c_double)

    def _with_mode(self, mode):
        q = _Params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(self._p), ctypes.sizeof(_Params))
        if mode is not None:
            q.mask_mode = MASK_MODES[mode]
        if q.mask_mode == MASK_MODES["teno6"]:
            self._attach_teno(q)
        return q

    def mask_size(self):
        n = self.nv * self.ny * (self.nx + 1)
        if self.ndim == 2:
            n += self.nv * (self.ny + 1) * self.nx
        return n

    def shape(self):
        return (self.nv, self.ny, self.nx)

    # -- the method ----------------------------------------------------------
    def rhs(self, U, mask_mode=None, mask_in=None, want_mask=False):
        lib = _load()
        U = _f64(U).reshape(self.shape())
        out = np.empty_like(U)
        q = self._with_mode("given" if mask_in is not None else mask_mode)
        mi = None if mask_in is None else np.ascontiguousarray(mask_in, dtype=np.uint8)
        mo = np.zeros(self.mask_size(), dtype=np.uint8) if want_mask else None
        bad = lib.oracle_rhs(ctypes.byref(q), _ptr(U, ctypes.c_double),
                             _ptr(out, ctypes.c_double), _ptr(mi, ctypes.c_uint8),
                             _ptr(mo, ctypes.c_uint8))
        self.last_nonphysical = bool(bad)
        return (out, mo) if want_mask else out

    def rhs_cells(self, U, cells, mask_mode=None):
        lib = _load()
        U = _f64(U).reshape(self.shape())
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((cells.size, self.nv), dtype=np.float64)
        q = self._with_mode(mask_mode)
        lib.oracle_rhs_cells(ctypes.byref(q), _ptr(U, ctypes.c_double), cells.size,
                             _ptr(cells, ctypes.c_int64), _ptr(out, ctypes.c_double))
        return out

    def face_masks(self, U, dirs, faces, lines, mask_mode=None):
        lib = _load()
        U = _f64(U).reshape(self.shape())
        dirs = np.ascontiguousarray(dirs, dtype=np.int32)
        faces = np.ascontiguousarray(faces, dtype=np.int32)
        lines = np.ascontiguousarray(lines, dtype=np.int32)
        out = np.zeros((dirs.size, self.nv), dtype=np.uint8)
        q = self._with_mode(mask_mode)
        lib.oracle_face_masks(ctypes.byref(q), _ptr(U, ctypes.c_double), dirs.size,
                              _ptr(dirs, ctypes.c_int32), _ptr(faces, ctypes.c_int32),
                              _ptr(lines, ctypes.c_int32), _ptr(out, ctypes.c_uint8))
        return out

    def jvp(self, U, V, mask):
        lib = _load()
        U = _f64(U).reshape(self.shape())
        V = _f64(V).reshape(self.shape())
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        f = np.empty_like(U)
        jv = np.empty_like(U)
        lib.oracle_rhs_jvp(ctypes.byref(self._p), _ptr(U, ctypes.c_double),
                           _ptr(V, ctypes.c_double), _ptr(mask, ctypes.c_uint8),
                           _ptr(f, ctypes.c_double), _ptr(jv, ctypes.c_double))
        return f, jv

    def jvp_cells(self, U, V, mask, cells):
        """(J V) at the listed cells (flat indices) only: [ncells][nv]."""
        lib = _load()
        U = _f64(U).reshape(self.shape())
        V = _f64(V).reshape(self.shape())
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((cells.size, self.nv), dtype=np.float64)
        lib.oracle_rhs_jvp_cells(ctypes.byref(self._p), _ptr(U, ctypes.c_double),
                                 _ptr(V, ctypes.c_double), _ptr(mask, ctypes.c_uint8),
                                 cells.size, _ptr(cells, ctypes.c_int64), _ptr(out, ctypes.c_double))
        return out

    def classify(self, X):
        lib = _load()
        X = _f64(X).reshape(-1, 6)
        eta = np.empty(X.shape[0], dtype=np.uint8)
        logits = np.empty((X.shape[0], 4), dtype=np.float64)
        lib.oracle_classify(ctypes.byref(self._p), _ptr(X, ctypes.c_double), X.shape[0],
                            _ptr(eta, ctypes.c_uint8), _ptr(logits, ctypes.c_double))
        return eta, logits

    def reconstruct(self, s, mask_mode="mlp", eta=0):
        lib = _load()
        s = _f64(s).reshape(6)
        e = np.array([eta], dtype=np.uint8)
        q = self._with_mode(mask_mode)
        v = lib.oracle_reconstruct(ctypes.byref(q), _ptr(s, ctypes.c_double),
                                   _ptr(e, ctypes.c_uint8))
        return v, int(e[0])

    def roe_eigen(self, direction, UL, UR):
        lib = _load()
        UL, UR = _f64(UL), _f64(UR)
        L = np.zeros(16)
        R = np.zeros(16)
        bad = lib.oracle_roe_eigen(ctypes.byref(self._p), direction, _ptr(UL, ctypes.c_double),
                                   _ptr(UR, ctypes.c_double), _ptr(L, ctypes.c_double),
                                   _ptr(R, ctypes.c_double))
        nv = self.nv
        return L.reshape(4, 4)[:nv, :nv], R.reshape(4, 4)[:nv, :nv], bad == 0

    def dt(self, U, cfl):
        U = _f64(U).reshape(self.shape())
        return _load().oracle_dt(ctypes.byref(self._p), _ptr(U, ctypes.c_double), cfl)

    def step(self, U, cfl, t=0.0, t_end=0.0):
        """One SSP-RK3 step; returns (U_new, t_new, dt)."""
        lib = _load()
        U = _f64(U).reshape(self.shape()).copy()
        tt = np.array([t], dtype=np.float64)
        dt = np.zeros(1)
        lib.oracle_step(ctypes.byref(self._p), _ptr(U, ctypes.c_double), cfl,
                        _ptr(tt, ctypes.c_double), t_end, _ptr(dt, ctypes.c_double))
        return U, float(tt[0]), float(dt[0])

    def scalar_solve(self, law, u0, cfl, t_end, mask_mode=None):
        """1D periodic scalar law (0 advection, 1 Burgers) to t_end."""
        lib = _load()
        u = _f64(u0).copy()
        assert u.size == self.nx
        q = self._with_mode(mask_mode)
        ns = np.zeros(1, dtype=np.int64)
        lib.oracle_scalar_solve(ctypes.byref(q), law, _ptr(u, ctypes.c_double), cfl, t_end,
                                _ptr(ns, ctypes.c_int64))
        return u, int(ns[0])
