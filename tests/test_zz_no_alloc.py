"""neno6_step_noalloc against neno6_step, through the C ABI.

The allocation-free step serves callers that cannot call cudaMalloc (a host
application that owns the GPU's memory through its own pool or budget, or a
latency-critical loop that must not be stalled by the device-wide
synchronisation of cudaMalloc/cudaFree).  It keeps its scratch in a static
device array shared by every call, so it is checked over two calls in a row:
the second call sees the first call's leftovers and must still match.  This
file is collected last on purpose.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

from conftest import balanced_net

import synth

pytestmark = pytest.mark.gpu

REL_L1_TOL = 1e-12  # the FP64 parity tolerance used throughout the tests
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def _cfg(p, ndim, nx, ny, bc="periodic"):
    c = p._Config()
    c.ndim, c.nx, c.ny = ndim, nx, ny
    c.dx, c.dy, c.gamma = 1.0 / nx, 1.0 / ny, 1.4
    c.bc[0] = c.bc[1] = p.BC[bc]
    c.precision, c.linear_weights, c.mask_mode = 0, 0, 0
    return c


def _noalloc(p, cfg, params, U, t=None, dt=None, status=None, t_end=0.0):
    ptr = lambda x: None if x is None else ctypes.c_void_p(x.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return p.load_library().neno6_step_noalloc(
        ctypes.byref(cfg), params.ctypes.data_as(ctypes.c_void_p), params.size, ptr(U), 0.4, t_end,
        ptr(t), ptr(dt), ptr(status), stream)


def _net(tmp_path, seed):
    net = balanced_net(seed)
    path = tmp_path / ("net%d.bin" % seed)
    net.save(path)
    return str(path), np.ascontiguousarray(net.packed(), dtype=np.float64)


def test_step_noalloc_matches_step_twice(lib, tmp_path):
    path, params = _net(tmp_path, 21)
    nx, ny = 40, 36
    U0 = synth.smooth_2d(nx, ny, seed=17)  # a random classifier stays stable on smooth data
    ref = lib.Neno6(ndim=2, nx=nx, ny=ny, weights=path)
    U_ref = torch.from_numpy(U0).cuda()
    U_new = torch.from_numpy(U0).cuda()
    t_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    t_new = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_new = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = _cfg(lib, 2, nx, ny)
    for call in range(2):
        ref.step(U_ref, 0.4, t=t_ref)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _noalloc(lib, cfg, params, U_new, t=t_new, dt=dt_new, status=status)
        assert rc == 0
        torch.cuda.synchronize()
        if call == 1:
            # the second call finds every kernel and the static array loaded:
            # the device's free memory must not move
            assert torch.cuda.mem_get_info()[0] == free_before
        a, b = U_new.cpu().numpy(), U_ref.cpu().numpy()
        assert np.isfinite(b).all()
        assert np.abs(a - b).sum() <= REL_L1_TOL * np.abs(b).sum(), call
        assert t_new.item() == t_ref.item() and dt_new.item() > 0.0
    assert status.item() == 0
    ref.close()


def test_step_noalloc_null_outputs_and_1d_transmissive(lib, tmp_path):
    """With t, dt and status all NULL the step starts from t = 0 and keeps its
    time and status words in the shared array (cleared by every call); a 1D
    transmissive Riemann state (the trained classifier, which keeps it
    physical), two calls in a row, each against one neno6_step of a fresh
    handle from t = 0."""
    from oracle.weights import Net
    path = os.path.join(ROOT, "weights", "neno6_mlp_6x64x32x16x8x4.bin")
    params = np.ascontiguousarray(Net.load(path).packed(), dtype=np.float64)
    n = 200
    U0 = synth.riemann_1d(n, seed=23)
    cfg = _cfg(lib, 1, n, 1, bc="transmissive")
    U_new = torch.from_numpy(U0).cuda()
    for call in range(2):
        start = U_new.clone()
        ref = lib.Neno6(ndim=1, nx=n, bc=("transmissive", "transmissive"), weights=path)
        U_ref = start.clone()
        ref.step(U_ref, 0.4, t_end=0.05)
        assert _noalloc(lib, cfg, params, U_new, t_end=0.05) == 0
        torch.cuda.synchronize()
        a, b = U_new.cpu().numpy(), U_ref.cpu().numpy()
        assert np.isfinite(b).all() and not np.array_equal(b, start.cpu().numpy())
        assert np.abs(a - b).sum() <= REL_L1_TOL * np.abs(b).sum(), call
        assert ref.status() == 0
        ref.close()


def test_step_noalloc_rejects_oversized_state(lib):
    params = np.zeros(3228)
    cfg = _cfg(lib, 2, 512, 512)  # 4 * 512 * 512 > the static scratch
    U = torch.zeros((4, 512, 512), dtype=torch.float64, device="cuda")
    rc = _noalloc(lib, cfg, params, U)
    assert rc == -2  # NENO6_ERR_SHAPE, nothing launched
