"""The mixed-precision path's difference and SSP-RK3 stage update (Eq.
(approximateEq), Sec. 4.4): the face kernel writes every face flux once and
the difference kernel forms each cell's difference and stage update.

* Determinism: repeated RHS evaluations and steps agree bit for bit
  (periodic, transmissive and mixed boundaries, ragged grids, 1D).
* The step equals three RHS evaluations combined on the host with the
  Shu-Osher weights (U1 = U + dt L(U), U2 = 3/4 U + 1/4 (U1 + dt L(U1)),
  U3 = 1/3 U + 2/3 (U2 + dt L(U2))): the stage update uses the right state,
  weights and dt, and t advances by dt.
"""
import numpy as np
import pytest
import torch

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


GRIDS = [(1024, 1024, ("periodic", "periodic")),
         (333, 257, ("transmissive", "transmissive")),
         (256, 97, ("periodic", "transmissive")),
         (48, 32, ("transmissive", "periodic"))]


@pytest.mark.parametrize("nx,ny,bc", GRIDS)
def test_rhs_and_step_bitwise_repeatable(lib, nx, ny, bc):
    g = lib.Neno6(ndim=2, nx=nx, ny=ny, bc=bc, precision="fp16")
    U = torch.from_numpy(synth.quadrants_2d(nx, ny, seed=21)).cuda()
    first = g.rhs(U)
    for _ in range(4):
        assert torch.equal(g.rhs(U), first)
    states = []
    for _ in range(3):
        V = U.clone()
        for _ in range(2):
            g.step(V, 0.4)
        states.append(V)
    assert torch.equal(states[0], states[1]) and torch.equal(states[0], states[2])
    assert g.status() == 0


def test_rhs_1d_repeatable(lib):
    g = lib.Neno6(ndim=1, nx=400, bc=("transmissive", "transmissive"), precision="fp16")
    U = torch.from_numpy(synth.riemann_1d(400, seed=3)).cuda()
    first = g.rhs(U)
    for _ in range(4):
        assert torch.equal(g.rhs(U), first)


@pytest.mark.parametrize("nx,ny,bc", GRIDS[1:])
def test_step_is_three_rhs_with_shu_osher_weights(lib, nx, ny, bc):
    g = lib.Neno6(ndim=2, nx=nx, ny=ny, bc=bc, precision="fp16")
    U0 = torch.from_numpy(synth.quadrants_2d(nx, ny, seed=22)).cuda()
    V = U0.clone()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.step(V, 0.4, t=t, dt=dt)
    h = dt.item()
    assert h > 0 and t.item() == h
    u0 = U0.cpu().numpy()
    u1 = u0 + h * g.rhs(U0).cpu().numpy()
    w = torch.from_numpy(u1).cuda()
    u2 = 0.75 * u0 + 0.25 * (u1 + h * g.rhs(w).cpu().numpy())
    w = torch.from_numpy(u2).cuda()
    u3 = u0 / 3.0 + 2.0 / 3.0 * (u2 + h * g.rhs(w).cpu().numpy())
    got = V.cpu().numpy()
    # the host rounds each combination differently from the kernel's FMAs,
    # and a one-ulp change of a stage state can move the FP32 rounding of a
    # cell's deviation from its block reference (relative 6e-8 of a
    # deviation of order |U|), i.e. the next RHS by up to ~1e-7 |L| and the
    # state by ~dt 1e-7 |L| <= 1e-10 |U|; a wrong weight, state or dt would
    # miss by O(dt |L|) ~ 1e-3 |U|
    scale = np.abs(u0).max(axis=(1, 2), keepdims=True)
    err = np.abs(got - u3) / scale
    print("step vs host combination of three RHS: max rel %.3e" % err.max())
    assert err.max() < 1e-10
