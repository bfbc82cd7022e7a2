"""The 1D Riemann workload run in full on the GPU against the FP64 oracle.

2 x 400 uniform cells on [0, 1], gamma = 1.4, transmissive boundaries,
seeded Riemann data (left/right rho in [0.1, 1], u in [-0.5, 0.5], p in
[0.1, 1], jump at x = 0.5), FP64 NENO6 with the trained classifier,
SSP-RK3 at CFL 0.5 to t = 0.2 (Sec. 4.4): every step's dt, time and state
must equal the oracle's bit for bit, and the classifier masks of the
evolving state are compared at regular intervals and at the end.
"""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "weights", "neno6_mlp_6x64x32x16x8x4.bin")


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def test_riemann_1d_400_to_t_0p2_bit_exact(lib, oracle_mod):
    from oracle.weights import Net
    n, cfl, t_end = 400, 0.5, 0.2
    bc = ("transmissive", "transmissive")
    o = oracle_mod.Oracle(ndim=1, nx=n, bc=bc, net=Net.load(WEIGHTS))
    g = lib.Neno6(ndim=1, nx=n, bc=bc, weights=WEIGHTS)
    U = synth.riemann_1d(n)
    Ug = torch.from_numpy(U.copy()).cuda()
    t_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    t, steps, masks_checked = 0.0, 0, 0
    while t < t_end:
        U, t, dt = o.step(U, cfl, t, t_end)
        g.step(Ug, cfl, t_end, t=t_dev, dt=dt_dev)
        steps += 1
        assert dt_dev.item() == dt and t_dev.item() == t, steps
        assert np.array_equal(Ug.cpu().numpy(), U), "state differs at step %d" % steps
        if steps % 50 == 0 or t >= t_end:
            d_o, m_o = o.rhs(U, want_mask=True)
            d_g, m_g = g.rhs(Ug, want_mask=True)
            assert np.array_equal(m_g.cpu().numpy(), m_o), "masks differ at step %d" % steps
            assert np.array_equal(d_g.cpu().numpy(), d_o)
            masks_checked += 1
    assert t == t_end and steps > 300 and masks_checked >= 6
    assert g.status() == 0 and np.isfinite(U).all()
    # the discontinuities are still there: the classifier discards stencils
    assert np.unpackbits(m_o).sum() > 0
    g.close()
