"""neno6_step_host: the SSP-RK3 step on a state in host memory gives the same
bits as neno6_step on the device, with the caller's time in and out."""
import numpy as np
import pytest
import torch

from conftest import balanced_net

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


@pytest.fixture(scope="module")
def wpath(tmp_path_factory):
    path = tmp_path_factory.mktemp("w") / "net.bin"
    balanced_net(7).save(path)
    return str(path)


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("nx,ny,bc", [(96, 72, ("periodic", "periodic")),
                                      # the mixed path's last stage then runs in 7 row bands
                                      # (6 x 80 rows + 45), copied out band by band
                                      (136, 525, ("periodic", "periodic")),
                                      (72, 1024, ("transmissive", "transmissive"))])
def test_step_host_matches_device_step(lib, wpath, prec, pinned, nx, ny, bc):
    if prec == "fp64" and ny > 100:
        pytest.skip("the FP64 path does not band; one size covers it")
    # the random test network keeps small states physical; the larger ones
    # take the trained network (the random one is dense in near-zero logits
    # and its rough decisions can drive the quadrant state unphysical)
    g = lib.Neno6(ndim=2, nx=nx, ny=ny, bc=bc, precision=prec,
                  weights=wpath if ny <= 100 else lib.DEFAULT_WEIGHTS)
    U0 = synth.quadrants_2d(nx, ny, seed=21)
    Ud = torch.from_numpy(U0.copy()).cuda()
    t_dev = torch.full((1,), 0.25, dtype=torch.float64, device="cuda")
    host = torch.from_numpy(U0.copy())
    if pinned:
        host = host.pin_memory()
    for _ in range(2):
        g.step(Ud, 0.4, t=t_dev)
    out, t = g.step_host(host, 0.4, t=0.25)
    out, t = g.step_host(out, 0.4, t=t, out=out)  # in place on the host array
    assert torch.equal(out, Ud.cpu())
    assert t == t_dev.item()
    assert np.array_equal(host.numpy(), U0)  # the input array is only read
    assert g.status() == 0


def test_step_host_clips_to_t_end(lib, wpath):
    g = lib.Neno6(ndim=2, nx=64, ny=48, precision="fp64", weights=wpath)
    host = torch.from_numpy(synth.quadrants_2d(64, 48, seed=22))
    t_end = 1e-5
    out, t = g.step_host(host, 0.4, t_end=t_end, t=0.5 * t_end)
    assert t == t_end
    ref = torch.from_numpy(synth.quadrants_2d(64, 48, seed=22)).cuda()
    t_dev = torch.full((1,), 0.5 * t_end, dtype=torch.float64, device="cuda")
    g.step(ref, 0.4, t_end=t_end, t=t_dev)
    assert torch.equal(out, ref.cpu())


def test_step_host_1d_mixed(lib):
    """1D mixed-precision handle: one band, copies in and out around it."""
    g = lib.Neno6(ndim=1, nx=400, bc=("transmissive", "transmissive"), precision="fp16")
    U0 = synth.riemann_1d(400, seed=3)
    Ud = torch.from_numpy(U0.copy()).cuda()
    t_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.step(Ud, 0.5, t=t_dev)
    out, t = g.step_host(torch.from_numpy(U0.copy()).pin_memory(), 0.5, t=0.0)
    assert torch.equal(out, Ud.cpu())
    assert t == t_dev.item()
