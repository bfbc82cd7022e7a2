"""The TENO6-opt mask mode (Sec. 2.1-2.2, the paper's comparison scheme) of
the FP64 right-hand side against the FP64 oracle, through the C ABI: the
selection runs on the split characteristic fluxes in place of the
classifier, in the same canonical arithmetic order on both sides, so masks,
dU/dt and states are compared bit for bit (the FP64 form's tolerance,
relative L1 <= 1e-12, is asserted as well)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

REL_L1_TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def _pair(lib, oracle_mod, ndim, nx, ny, bc):
    g = lib.Neno6(ndim=ndim, nx=nx, ny=ny, bc=bc, mask_mode="teno6")
    o = oracle_mod.Oracle(ndim=ndim, nx=nx, ny=ny, bc=bc, mask_mode="teno6")
    return g, o


def _state(kind, ndim, nx, ny, seed):
    if kind == "quadrants":
        return synth.quadrants_2d(nx, ny, seed=seed)
    if kind == "smooth":
        return synth.smooth_2d(nx, ny, seed=seed)
    return synth.noisy(synth.riemann_1d(nx, seed=seed), seed=seed + 1, rel=0.02)


CASES = [
    (2, 40, 36, ("periodic", "periodic"), "quadrants"),       # several TMA tiles + ragged
    (2, 200, 136, ("periodic", "periodic"), "quadrants"),     # interior tiles by TMA
    (2, 33, 17, ("transmissive", "transmissive"), "quadrants"),
    (2, 64, 32, ("periodic", "transmissive"), "smooth"),
    (1, 400, 1, ("transmissive", "transmissive"), "riemann"),
]


@pytest.mark.parametrize("ndim,nx,ny,bc,kind", CASES)
def test_teno_rhs_parity(lib, oracle_mod, ndim, nx, ny, bc, kind):
    g, o = _pair(lib, oracle_mod, ndim, nx, ny, bc)
    U = _state(kind, ndim, nx, ny, seed=nx + ny)
    d_o, m_o = o.rhs(U, want_mask=True)
    d_g, m_g = g.rhs(torch.from_numpy(U).cuda(), want_mask=True)
    d_g, m_g = d_g.cpu().numpy(), m_g.cpu().numpy()
    assert g.status() == 0
    assert np.array_equal(m_g, m_o), "TENO6-opt masks differ"
    assert np.abs(d_g - d_o).sum() <= REL_L1_TOL * np.abs(d_o).sum()
    assert np.array_equal(d_g, d_o)
    if kind != "smooth":
        assert np.unpackbits(m_o).mean() > 0.005  # discontinuities: stencils discarded


def test_teno_step_parity(lib, oracle_mod):
    for ndim, n, ny, bc, kind, cfl in [(2, 48, 40, ("periodic", "periodic"), "quadrants", 0.4),
                                       (1, 400, 1, ("transmissive", "transmissive"), "riemann", 0.5)]:
        g, o = _pair(lib, oracle_mod, ndim, n, ny, bc)
        U = _state(kind, ndim, n, ny, seed=3)
        Ug = torch.from_numpy(U.copy()).cuda()
        t_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        t = 0.0
        for _ in range(4):
            U, t, _ = o.step(U, cfl, t, 0.0)
            g.step(Ug, cfl, t=t_dev)
            assert t_dev.item() == t
            assert np.array_equal(Ug.cpu().numpy(), U)
        assert g.status() == 0


def test_teno_full_size_sampled(lib, oracle_mod):
    """2048^2 periodic four-quadrant workload: sampled cells (dU/dt) and
    faces (masks) against the oracle one by one."""
    n = 2048
    g, o = _pair(lib, oracle_mod, 2, n, n, ("periodic", "periodic"))
    U = synth.quadrants_2d(n, n)
    d_g, m_g = g.rhs(torch.from_numpy(U).cuda(), want_mask=True)
    d_g, m_g = d_g.cpu().numpy(), m_g.cpu().numpy()
    rng = np.random.default_rng(7)
    cells = np.concatenate([rng.integers(0, n * n, 200), [0, n - 1, n * (n - 1), n * n - 1,
                                                          (n // 2) * n + n // 2]])
    assert np.array_equal(d_g.reshape(4, -1)[:, cells].T, o.rhs_cells(U, cells, mask_mode="teno6"))
    k = 150
    dirs, faces, lines = rng.integers(0, 2, k), rng.integers(0, n + 1, k), rng.integers(0, n, k)
    ref_m = o.face_masks(U, dirs, faces, lines, mask_mode="teno6")
    xblock = 4 * n * (n + 1)
    for r in range(k):
        for m in range(4):
            if dirs[r] == 0:
                idx = (m * n + lines[r]) * (n + 1) + faces[r]
            else:
                idx = xblock + (m * (n + 1) + faces[r]) * n + lines[r]
            assert m_g[idx] == ref_m[r, m]
