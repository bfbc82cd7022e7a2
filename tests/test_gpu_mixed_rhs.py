"""Mixed-precision right-hand side and RK3 step against the FP64 path.

The FP64 path is bit-exact with the oracle (test_gpu_parity.py), so it is the
reference here.  With the classifier switched off (all stencils kept, or all
discarded) only the FP32 reconstruction arithmetic differs, and the error
must stay at FP32 level; with the classifier on, the bf16/fp16 decisions may
flip a few stencils, which the mask comparison counts.
"""
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
    balanced_net(41).save(path)
    return str(path)


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def pair(lib, wpath, prec, **kw):
    return (lib.Neno6(precision="fp64", weights=wpath, **kw),
            lib.Neno6(precision=prec, weights=wpath, **kw))


@pytest.mark.parametrize("mode", ["smooth", "rough"])
@pytest.mark.parametrize("ndim,nx,ny,bc", [(2, 200, 136, ("periodic", "periodic")),
                                           (2, 67, 33, ("transmissive", "transmissive")),
                                           (1, 400, 1, ("transmissive", "transmissive"))])
def test_mixed_reconstruction_arithmetic(lib, wpath, mode, ndim, nx, ny, bc):
    """Classifier off: the only difference is FP32 reconstruction."""
    g64, gmx = pair(lib, wpath, "bf16", ndim=ndim, nx=nx, ny=ny, bc=bc, mask_mode=mode)
    U = (synth.quadrants_2d(nx, ny, seed=3) if ndim == 2
         else synth.noisy(synth.riemann_1d(nx, seed=3), seed=4, rel=0.02))
    Ud = torch.from_numpy(U).cuda()
    d64, m64 = g64.rhs(Ud, want_mask=True)
    dmx, mmx = gmx.rhs(Ud, want_mask=True)
    assert torch.equal(m64, mmx)
    d64, dmx = d64.cpu().numpy(), dmx.cpu().numpy()
    err = rel_l1(dmx, d64)
    print("rel L1 (%s, %s) = %.3e" % (mode, (ndim, nx, ny), err))
    assert err < 2e-5
    assert gmx.status() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mixed_rhs_with_classifier(lib, wpath, prec):
    nx, ny = 200, 136
    g64, gmx = pair(lib, wpath, prec, ndim=2, nx=nx, ny=ny)
    U = synth.quadrants_2d(nx, ny, seed=5)
    Ud = torch.from_numpy(U).cuda()
    d64, m64 = g64.rhs(Ud, want_mask=True)
    dmx, mmx = gmx.rhs(Ud, want_mask=True)
    m64, mmx = m64.cpu().numpy(), mmx.cpu().numpy()
    flips = np.unpackbits(m64 ^ mmx).sum() / (8.0 * m64.size)
    err = rel_l1(dmx.cpu().numpy(), d64.cpu().numpy())
    print("%s: flip rate %.3e, rel L1 %.3e" % (prec, flips, err))
    assert flips < 2e-3
    assert err < 1e-2


def test_mixed_constant_state_and_conservation(lib, wpath):
    _, gmx = pair(lib, wpath, "bf16", ndim=2, nx=96, ny=80)
    U = synth.prim_to_cons(np.full((80, 96), 0.7), 0.3, -0.2, 1.1)
    assert torch.count_nonzero(gmx.rhs(torch.from_numpy(U).cuda())).item() == 0
    U = synth.quadrants_2d(96, 80, seed=6)
    d = gmx.rhs(torch.from_numpy(U).cuda()).cpu().numpy()
    assert np.all(np.abs(d.sum(axis=(1, 2))) <= 1e-12 * np.abs(d).sum(axis=(1, 2)))


def test_mixed_step_close_to_fp64(lib, wpath):
    nx = ny = 128
    g64, gmx = pair(lib, wpath, "bf16", ndim=2, nx=nx, ny=ny, mask_mode="smooth")
    U = synth.smooth_2d(nx, ny, seed=9)
    A = torch.from_numpy(U).cuda()
    B = torch.from_numpy(U).cuda()
    ta = torch.zeros(1, dtype=torch.float64, device="cuda")
    tb = torch.zeros(1, dtype=torch.float64, device="cuda")
    dta = torch.zeros(1, dtype=torch.float64, device="cuda")
    dtb = torch.zeros(1, dtype=torch.float64, device="cuda")
    for step in range(3):
        g64.step(A, 0.4, t=ta, dt=dta)
        gmx.step(B, 0.4, t=tb, dt=dtb)
        # the mixed path's wave-speed maximum takes velocities and sound
        # speed in FP32 (pressure in FP64): dt agrees to FP32 rounding
        assert abs(dta.item() - dtb.item()) <= 1e-6 * dta.item()
    err = rel_l1(B.cpu().numpy(), A.cpu().numpy())
    print("state rel L1 after 3 steps: %.3e" % err)
    assert err < 1e-6
    assert abs(ta.item() - tb.item()) <= 1e-6 * ta.item()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,bc", [(200, 136, ("periodic", "periodic")),
                                      (67, 33, ("transmissive", "transmissive"))])
def test_mixed_rhs_trained_network_bounds(lib, prec, nx, ny, bc):
    """The trained classifier (default weights, default guard bands) at the
    parity sizes, held to the mixed-precision targets: decision flip rate at
    most 1e-5 and dU/dt within 1e-6 relative L1 of the FP64 path (the
    random network above is dense in near-zero logits and pins little)."""
    g64 = lib.Neno6(precision="fp64", ndim=2, nx=nx, ny=ny, bc=bc)
    gmx = lib.Neno6(precision=prec, ndim=2, nx=nx, ny=ny, bc=bc)
    Ud = torch.from_numpy(synth.quadrants_2d(nx, ny, seed=5)).cuda()
    d64, m64 = g64.rhs(Ud, want_mask=True)
    dmx, mmx = gmx.rhs(Ud, want_mask=True)
    m64, mmx = m64.cpu().numpy(), mmx.cpu().numpy()
    flips = np.unpackbits(m64 ^ mmx).sum() / (8.0 * m64.size)
    err = rel_l1(dmx.cpu().numpy(), d64.cpu().numpy())
    print("trained %s %dx%d: flip rate %.3e, rel L1 %.3e" % (prec, nx, ny, flips, err))
    assert flips <= 1e-5
    assert err <= 1e-6
    assert gmx.status() == 0
