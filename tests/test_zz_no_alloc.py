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

import numpy as np
import pytest
import torch

from conftest import balanced_net

import synth

pytestmark = pytest.mark.gpu

REL_L1_TOL = 1e-12  # the FP64 parity tolerance used throughout the tests


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def _cfg(p, ndim, nx, ny):
    c = p._Config()
    c.ndim, c.nx, c.ny = ndim, nx, ny
    c.dx, c.dy, c.gamma = 1.0 / nx, 1.0 / ny, 1.4
    c.bc[0] = c.bc[1] = p.BC["periodic"]
    c.precision, c.linear_weights, c.mask_mode = 0, 0, 0
    return c


def test_step_noalloc_matches_step_twice(lib, tmp_path):
    net = balanced_net(21)
    path = tmp_path / "net.bin"
    net.save(path)
    params = np.ascontiguousarray(net.packed(), dtype=np.float64)
    nx, ny = 40, 36
    U0 = synth.smooth_2d(nx, ny, seed=17)  # a random classifier stays stable on smooth data
    ref = lib.Neno6(ndim=2, nx=nx, ny=ny, weights=str(path))
    U_ref = torch.from_numpy(U0).cuda()
    U_new = torch.from_numpy(U0).cuda()
    t_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    t_new = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_new = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = _cfg(lib, 2, nx, ny)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        ref.step(U_ref, 0.4, t=t_ref)
        rc = lib.load_library().neno6_step_noalloc(
            ctypes.byref(cfg), params.ctypes.data_as(ctypes.c_void_p), params.size,
            ctypes.c_void_p(U_new.data_ptr()), 0.4, 0.0, ctypes.c_void_p(t_new.data_ptr()),
            ctypes.c_void_p(dt_new.data_ptr()), ctypes.c_void_p(status.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        a, b = U_new.cpu().numpy(), U_ref.cpu().numpy()
        assert np.isfinite(b).all()
        assert np.abs(a - b).sum() <= REL_L1_TOL * np.abs(b).sum(), call
        assert t_new.item() == t_ref.item() and dt_new.item() > 0.0
    assert status.item() == 0
    ref.close()


def test_step_noalloc_rejects_oversized_state(lib):
    params = np.zeros(3228)
    cfg = _cfg(lib, 2, 512, 512)  # 4 * 512 * 512 > the static scratch
    U = torch.zeros((4, 512, 512), dtype=torch.float64, device="cuda")
    rc = lib.load_library().neno6_step_noalloc(
        ctypes.byref(cfg), params.ctypes.data_as(ctypes.c_void_p), params.size,
        ctypes.c_void_p(U.data_ptr()), 0.4, 0.0, None, None, None, None)
    assert rc == -2  # NENO6_ERR_SHAPE, nothing launched
