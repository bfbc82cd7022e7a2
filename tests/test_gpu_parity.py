"""Parity of the CUDA FP64 path with the FP64 oracle, through the C ABI.

The FP64 path evaluates every quantity in the same order as the oracle, so
the expectation is bit-exact classifier masks (required of the FP64 form)
and bit-exact states; the state tolerance written in the tests is the FP64
form's relative L1 <= 1e-12, with the exact-match count asserted
separately.
"""
import numpy as np
import pytest
import torch

from conftest import balanced_net

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


@pytest.fixture(scope="module")
def net_file(tmp_path_factory):
    net = balanced_net(11)
    path = tmp_path_factory.mktemp("w") / "net.bin"
    net.save(path)
    return net, str(path)


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def make_pair(lib, oracle_mod, net_file, ndim, nx, ny, bc, **kw):
    net, path = net_file
    g = lib.Neno6(ndim=ndim, nx=nx, ny=ny, bc=bc, weights=path, **kw)
    o = oracle_mod.Oracle(ndim=ndim, nx=nx, ny=ny, bc=bc, net=net, **kw)
    return g, o


def to_dev(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


# ------------------------------------------------------------------ classify
def test_classify_bit_exact(lib, oracle_mod, net_file):
    g, o = make_pair(lib, oracle_mod, net_file, 1, 8, 1, ("periodic", "periodic"))
    X = synth.mlp_stencils(20000, seed=5)
    # adversarial rows: scaled copies straddling max|s| = 1, tiny values
    X = np.concatenate([X, X[:2000] * 1e-3, X[:2000] / np.abs(X[:2000]).max(1, keepdims=True)])
    eta_o, z_o = o.classify(X)
    eta_g, z_g = g.classify(to_dev(X), want_logits=True)
    assert np.array_equal(eta_g.cpu().numpy(), eta_o)
    assert np.array_equal(z_g.cpu().numpy(), z_o)
    assert 0.1 < np.unpackbits(eta_o).mean() * 2 < 0.9  # both outcomes exercised


def test_classify_empty_and_odd_sizes(lib, oracle_mod, net_file):
    g, o = make_pair(lib, oracle_mod, net_file, 1, 8, 1, ("periodic", "periodic"))
    for n in (0, 1, 255, 257):
        X = synth.mlp_stencils(max(n, 2), seed=n)[:n]
        eta = g.classify(to_dev(X) if n else torch.empty((0, 6), dtype=torch.float64, device="cuda"))
        if n:
            assert np.array_equal(eta.cpu().numpy(), o.classify(X)[0])
        else:
            assert eta.numel() == 0


# ----------------------------------------------------------------------- RHS
CASES = [
    # ndim, nx, ny, bc, generator
    (2, 40, 36, ("periodic", "periodic"), "quadrants"),      # several tiles + ragged
    (2, 33, 17, ("transmissive", "transmissive"), "quadrants"),
    (2, 64, 32, ("periodic", "transmissive"), "smooth"),
    (2, 5, 3, ("periodic", "periodic"), "quadrants"),        # grid smaller than the halo
    (1, 400, 1, ("transmissive", "transmissive"), "riemann"),  # the 1D Riemann workload
    (1, 130, 1, ("periodic", "periodic"), "riemann"),
    (1, 2, 1, ("periodic", "periodic"), "riemann"),
]


def _state(kind, ndim, nx, ny, seed):
    if kind == "quadrants":
        return synth.quadrants_2d(nx, ny, seed=seed)
    if kind == "smooth":
        return synth.smooth_2d(nx, ny, seed=seed)
    return synth.noisy(synth.riemann_1d(nx, seed=seed), seed=seed + 1, rel=0.02)


@pytest.mark.parametrize("ndim,nx,ny,bc,kind", CASES)
def test_rhs_parity(lib, oracle_mod, net_file, ndim, nx, ny, bc, kind):
    g, o = make_pair(lib, oracle_mod, net_file, ndim, nx, ny, bc)
    U = _state(kind, ndim, nx, ny, seed=nx + ny)
    d_o, m_o = o.rhs(U, want_mask=True)
    d_g, m_g = g.rhs(to_dev(U), want_mask=True)
    d_g, m_g = d_g.cpu().numpy(), m_g.cpu().numpy()
    assert g.status() == 0
    assert np.array_equal(m_g, m_o), "classifier masks differ"
    assert rel_l1(d_g, d_o) <= REL_L1_TOL
    assert np.array_equal(d_g, d_o), "FP64 path is expected to be bit-identical"
    bits = np.unpackbits(m_o)
    assert 0.05 < bits.mean() < 0.95


@pytest.mark.parametrize("mode", ["smooth", "rough"])
def test_rhs_mask_modes(lib, oracle_mod, net_file, mode):
    g, o = make_pair(lib, oracle_mod, net_file, 2, 40, 20, ("periodic", "periodic"), mask_mode=mode)
    U = synth.quadrants_2d(40, 20, seed=3)
    d_o, m_o = o.rhs(U, want_mask=True)
    d_g, m_g = g.rhs(to_dev(U), want_mask=True)
    assert np.array_equal(m_g.cpu().numpy(), m_o)
    assert np.array_equal(d_g.cpu().numpy(), d_o)


def test_rhs_frozen_mask(lib, oracle_mod, net_file):
    g, o = make_pair(lib, oracle_mod, net_file, 2, 34, 18, ("periodic", "periodic"))
    U = synth.quadrants_2d(34, 18, seed=4)
    rng = np.random.default_rng(0)
    mask = rng.integers(0, 256, o.mask_size(), dtype=np.uint8)
    d_o = o.rhs(U, mask_in=mask)
    d_g, m_g = g.rhs(to_dev(U), mask_in=torch.from_numpy(mask).cuda(), want_mask=True)
    assert np.array_equal(m_g.cpu().numpy(), mask)
    assert np.array_equal(d_g.cpu().numpy(), d_o)


def test_rhs_sixth_order_weights(lib, oracle_mod, net_file):
    g, o = make_pair(lib, oracle_mod, net_file, 2, 32, 32, ("periodic", "periodic"),
                     linear_weights="sixth")
    U = synth.smooth_2d(32, 32, seed=8)
    assert np.array_equal(g.rhs(to_dev(U)).cpu().numpy(), o.rhs(U))


def test_constant_state_and_conservation_on_gpu(lib, oracle_mod, net_file):
    g, _ = make_pair(lib, oracle_mod, net_file, 2, 48, 40, ("periodic", "periodic"))
    U = synth.prim_to_cons(np.full((40, 48), 0.9), 0.2, -0.4, 1.1)
    assert torch.count_nonzero(g.rhs(to_dev(U))).item() == 0
    U = synth.quadrants_2d(48, 40, seed=9)
    d = g.rhs(to_dev(U)).cpu().numpy()
    assert np.all(np.abs(d.sum(axis=(1, 2))) <= 1e-13 * np.abs(d).sum(axis=(1, 2)))


# ---------------------------------------------------------------------- step
@pytest.mark.parametrize("ndim,nx,ny,bc,kind,t_end",
                         [(2, 40, 36, ("periodic", "periodic"), "quadrants", 0.0),
                          (1, 400, 1, ("transmissive", "transmissive"), "riemann", 0.0),
                          (1, 100, 1, ("transmissive", "transmissive"), "riemann", 0.004)])
def test_step_parity(lib, oracle_mod, net_file, ndim, nx, ny, bc, kind, t_end):
    g, o = make_pair(lib, oracle_mod, net_file, ndim, nx, ny, bc)
    U = _state(kind, ndim, nx, ny, seed=7)
    Ug = to_dev(U)
    t_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = 0.0
    cfl = 0.5 if ndim == 1 else 0.4
    for _ in range(3):
        U, t, dt = o.step(U, cfl, t, t_end)
        g.step(Ug, cfl, t_end, t=t_dev, dt=dt_dev)
        assert dt_dev.item() == dt
        assert t_dev.item() == t
        assert np.array_equal(Ug.cpu().numpy(), U)
    assert g.status() == 0
    if t_end:
        assert t == t_end


# ---------------------------------------------------- full size, sampled
def test_full_size_sampled_parity(lib, oracle_mod, net_file):
    """2048^2 periodic four-quadrant workload in the benchmark's launch
    configuration: sampled cells and faces against the oracle, one by one."""
    n = 2048
    g, o = make_pair(lib, oracle_mod, net_file, 2, n, n, ("periodic", "periodic"))
    U = synth.quadrants_2d(n, n)
    d_g, m_g = g.rhs(to_dev(U), want_mask=True)
    d_g, m_g = d_g.cpu().numpy(), m_g.cpu().numpy()
    rng = np.random.default_rng(1)
    cells = rng.integers(0, n * n, 300)
    # include the four quadrant junctions and the periodic edges
    cells = np.concatenate([cells, [0, n - 1, n * (n - 1), n * n - 1, (n // 2) * n + n // 2,
                                    (n // 2 - 1) * n + n // 2 - 1]])
    ref = o.rhs_cells(U, cells)
    got = d_g.reshape(4, -1)[:, cells].T
    assert np.array_equal(got, ref)
    # masks of sampled faces
    k = 200
    dirs = rng.integers(0, 2, k)
    faces = rng.integers(0, n + 1, k)
    lines = rng.integers(0, n, k)
    ref_m = o.face_masks(U, dirs, faces, lines)
    xblock = 4 * n * (n + 1)
    for r in range(k):
        for m in range(4):
            if dirs[r] == 0:
                idx = (m * n + lines[r]) * (n + 1) + faces[r]
            else:
                idx = xblock + (m * (n + 1) + faces[r]) * n + lines[r]
            assert m_g[idx] == ref_m[r, m]


# -------------------------------------------------------------- error paths
def test_nonphysical_state_sets_status(lib, oracle_mod, net_file):
    g, _ = make_pair(lib, oracle_mod, net_file, 2, 16, 16, ("periodic", "periodic"))
    U = synth.quadrants_2d(16, 16, seed=2)
    U[3, 5, 7] = -1.0  # negative energy -> negative pressure
    g.rhs(to_dev(U))
    assert g.status() & 1
    assert g.status() == 0  # cleared


def test_bad_arguments_return_codes(lib, net_file):
    import ctypes
    _, path = net_file
    g = lib.Neno6(ndim=2, nx=8, ny=8, weights=path)
    U = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    rc = g._lib.neno6_rhs(g._h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                          None, None, None)
    assert rc == -1  # aliasing
    rc = g._lib.neno6_rhs(g._h, ctypes.c_void_p(U.data_ptr() + 8), ctypes.c_void_p(U.data_ptr()),
                          None, None, None)
    assert rc == -3  # misaligned
    with pytest.raises(lib.Neno6Error):
        lib.Neno6(ndim=2, nx=8, ny=8, weights=path, precision="fp64", gamma=0.5)
