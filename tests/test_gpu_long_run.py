"""The 2048^2 periodic four-quadrant workload over its ~100 SSP-RK3 steps
(to t = 0.0024, which the FP64 path reaches in 99 steps of CFL 0.4).

The FP64 path is checked against the oracle on the evolved state (the
quadrant interfaces have steepened into shocks and contacts by then): the
classifier bits of sampled faces and dU/dt at sampled cells, bit for bit.  Mass,
momentum and energy are conserved to round-off over the run.  The mixed path
(fp16 classifier) advanced from the same state to the same time stays within
the stated 1e-6 relative L1 of the FP64 path's state.  Each run takes its own
dt from its own state (near a shock a decision taken differently moves the
largest wave speed, and so dt, by ~1e-4 relative), so both runs clip their last
step to end exactly at t_end and the states are compared at equal times.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

N, T_END, CFL = 2048, 0.0024, 0.4


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def test_fp64_100_steps_against_oracle_and_mixed(lib, oracle_mod):
    from oracle.weights import Net
    U0 = synth.quadrants_2d(N, N)
    g = lib.Neno6(ndim=2, nx=N, ny=N)
    U = torch.from_numpy(U0).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    steps = 0
    while t.item() < T_END:
        g.step(U, CFL, t_end=T_END, t=t)
        steps += 1
    assert g.status() == 0 and t.item() == T_END and 90 <= steps <= 110
    Uh = U.cpu().numpy()
    # conservation on the periodic grid
    tot0, tot = U0.sum(axis=(1, 2)), Uh.sum(axis=(1, 2))
    assert np.all(np.abs(tot - tot0) <= 1e-12 * np.abs(U0).sum(axis=(1, 2)))
    # the FP64 path against the oracle on the evolved state
    d, m = g.rhs(U, want_mask=True)
    d, m = d.cpu().numpy(), m.cpu().numpy()
    o = oracle_mod.Oracle(ndim=2, nx=N, ny=N, net=Net.load(lib.DEFAULT_WEIGHTS))
    rng = np.random.default_rng(7)
    cells = rng.integers(0, N * N, 300)
    assert np.array_equal(d.reshape(4, -1)[:, cells].T, o.rhs_cells(Uh, cells))
    k = 300
    dirs = rng.integers(0, 2, k)
    faces = rng.integers(0, N + 1, k)
    lines = rng.integers(0, N, k)
    ref_m = o.face_masks(Uh, dirs, faces, lines)
    xblock = 4 * N * (N + 1)
    for r in range(k):
        for f in range(4):
            idx = ((f * N + lines[r]) * (N + 1) + faces[r] if dirs[r] == 0
                   else xblock + (f * (N + 1) + faces[r]) * N + lines[r])
            assert m[idx] == ref_m[r, f]
    # the mixed path over the same 100 steps
    gm = lib.Neno6(ndim=2, nx=N, ny=N, precision="fp16")
    V = torch.from_numpy(U0).cuda()
    tm = torch.zeros(1, dtype=torch.float64, device="cuda")
    steps_m = 0
    while tm.item() < T_END:
        gm.step(V, CFL, t_end=T_END, t=tm)
        steps_m += 1
    assert gm.status() == 0 and tm.item() == T_END
    err = ((V - U).abs().sum() / U.abs().sum()).item()
    errinf = ((V - U).abs().max() / U.abs().max()).item()
    print("t = %.4f: %d FP64 steps, %d mixed steps, state rel L1 %.2e, rel Linf %.2e"
          % (T_END, steps, steps_m, err, errinf))
    assert err <= 1e-6
