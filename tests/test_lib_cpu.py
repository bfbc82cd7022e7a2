"""Host-side checks of the CUDA library that need no GPU: it builds for
sm_103a, loads, and exports every entry point include/neno6.h declares."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib_path():
    from paper_2207_08500_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "neno6.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(neno6_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("neno6_rhs", "neno6_step", "neno6_classify"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    import paper_2207_08500_gb300 as p
    assert sorted(p.EXPORTS) == _declared()


def test_binding_declares_signatures_without_cuda(lib_path):
    import paper_2207_08500_gb300 as p
    lib = p.load_library(lib_path)
    assert lib.neno6_mask_bytes.restype is ctypes.c_int64
    # null handle: rejected without touching the device
    assert lib.neno6_mask_bytes(None) == -1
    assert lib.neno6_rhs(None, None, None, None, None, None) == -1
    assert lib.neno6_last_error(None) is not None


def test_create_rejects_bad_config_on_host(lib_path):
    import paper_2207_08500_gb300 as p
    lib = p.load_library(lib_path)
    c = p._Config()
    c.ndim, c.nx, c.ny, c.dx, c.dy, c.gamma = 3, 8, 8, 0.1, 0.1, 1.4
    h = ctypes.c_void_p()
    assert lib.neno6_create(ctypes.byref(c), b"/nonexistent", ctypes.byref(h)) == -1
    c.ndim, c.gamma = 2, 1.0
    assert lib.neno6_create(ctypes.byref(c), b"/nonexistent", ctypes.byref(h)) == -1
    c.gamma, c.nx = 1.4, 0
    assert lib.neno6_create(ctypes.byref(c), b"/nonexistent", ctypes.byref(h)) == -2
    c.nx = 8
    assert lib.neno6_create(ctypes.byref(c), b"/nonexistent", ctypes.byref(h)) == -4
    assert b"weights" in lib.neno6_last_error(None)


def test_solver_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2207_08500_gb300 as p
    with pytest.raises(RuntimeError):
        p.Neno6(ndim=1, nx=8)


def test_create_rejects_other_network_widths(lib_path, tmp_path):
    """The kernels are written for the 6-64-32-16-8-4 classifier of Sec. 3.1
    and, for neno6_classify, the width study's 6-32-32-32-4; a weights file of
    any other shape (here 6-32-16-4, and 6-64-32-16-4) is refused on the host
    with NENO6_ERR_WEIGHTS, before any device work."""
    import paper_2207_08500_gb300 as p
    from oracle.weights import Net
    lib = p.load_library(lib_path)
    c = p._Config()
    c.ndim, c.nx, c.ny, c.dx, c.dy, c.gamma = 2, 8, 8, 0.1, 0.1, 1.4
    for widths in [(6, 32, 16, 4), (6, 64, 32, 16, 4), (6, 32, 32, 16, 4)]:
        path = tmp_path / ("w%d.bin" % len(widths))
        Net.random(widths=widths, seed=3).save(path)
        h = ctypes.c_void_p()
        assert lib.neno6_create(ctypes.byref(c), str(path).encode(), ctypes.byref(h)) == -4
        assert b"6-64-32-16-8-4" in lib.neno6_last_error(None)


def test_create_refuses_teno6_mask_on_mixed_precision(lib_path):
    """The TENO6-opt mask mode runs on the FP64 path only: a mixed-precision
    handle with it is refused (NENO6_ERR_UNSUPPORTED) before any device work."""
    import paper_2207_08500_gb300 as p
    lib = p.load_library(lib_path)
    c = p._Config()
    c.ndim, c.nx, c.ny, c.dx, c.dy, c.gamma = 2, 8, 8, 0.1, 0.1, 1.4
    c.mask_mode = p.MASK_MODE["teno6"]
    for prec in ("bf16", "fp16"):
        c.precision = p.PRECISION[prec]
        h = ctypes.c_void_p()
        assert lib.neno6_create(ctypes.byref(c), b"/nonexistent", ctypes.byref(h)) == -8
        assert b"TENO6" in lib.neno6_last_error(None)
