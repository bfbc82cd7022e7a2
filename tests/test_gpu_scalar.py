"""Scalar conservation laws on the GPU (neno6_scalar_rhs / neno6_scalar_solve):
linear advection (Sec. 4.1) and Burgers (Sec. 4.2) with the NENO6
reconstruction, against the FP64 oracle (bit for bit) and against the
paper's Table "sinorder" (linear column, printed digits)."""
import math

import numpy as np
import pytest
import torch

from conftest import balanced_net, golden

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
def net_file(tmp_path_factory):
    net = balanced_net(21)
    path = tmp_path_factory.mktemp("w") / "net.bin"
    net.save(path)
    return net, str(path)


def _initial(n, kind, seed):
    x = (np.arange(n) + 0.5) / n
    rng = np.random.default_rng(seed)
    if kind == "sine":
        return np.sin(2 * math.pi * x) + 0.5 * np.sin(6 * math.pi * x + rng.uniform(0, 6))
    # square pulse plus a smooth bump: jumps of both signs
    return np.where((x > 0.2) & (x < 0.45), 1.0, -0.3) + 0.2 * np.exp(-((x - 0.75) / 0.05) ** 2)


@pytest.mark.parametrize("law", ["advection", "burgers"])
@pytest.mark.parametrize("mode", ["mlp", "smooth", "rough", "teno6"])
@pytest.mark.parametrize("n,bc,kind", [(400, "periodic", "sine"), (400, "transmissive", "pulse"),
                                       (37, "periodic", "pulse")])
def test_scalar_solve_bit_exact(lib, oracle_mod, net_file, law, mode, n, bc, kind):
    net, path = net_file
    if mode == "smooth" and kind == "pulse":
        pytest.skip("the unlimited linear scheme on a jump is not a meaningful case")
    g = lib.Neno6(ndim=1, nx=n, dx=1.0 / n, bc=(bc, bc), mask_mode=mode, weights=path)
    o = oracle_mod.Oracle(ndim=1, nx=n, dx=1.0 / n, bc=(bc, bc), net=net)
    u0 = _initial(n, kind, seed=n)
    t_end = 0.15 if law == "burgers" else 0.05  # Burgers: past the shock time of the sine data
    u = torch.from_numpy(u0.copy()).cuda()
    steps = g.scalar_solve(law, u, 0.4, t_end)
    ref, ref_steps = o.scalar_solve(0 if law == "advection" else 1, u0, 0.4, t_end, mask_mode=mode)
    assert steps == ref_steps
    assert np.array_equal(u.cpu().numpy(), ref)
    assert g.status() == 0


def test_scalar_rhs_first_order_upwind_when_all_discarded(lib, net_file):
    """Every stencil discarded, linear advection: the face flux is u_i exactly
    (g+ = u, g- = 0), so du/dt = -(u_i - u_{i-1}) / dx."""
    _, path = net_file
    n = 64
    g = lib.Neno6(ndim=1, nx=n, dx=1.0 / n, mask_mode="rough", weights=path)
    u0 = np.random.default_rng(3).normal(size=n)
    d, m = g.scalar_rhs("advection", torch.from_numpy(u0).cuda(), want_mask=True)
    assert np.array_equal(d.cpu().numpy(), -((u0 - np.roll(u0, 1)) / (1.0 / n)))
    assert np.all(m.cpu().numpy() == 0xFF)


def test_scalar_rhs_masks_and_conservation(lib, net_file):
    _, path = net_file
    n = 128
    g = lib.Neno6(ndim=1, nx=n, dx=1.0 / n, weights=path)
    u0 = _initial(n, "pulse", seed=5)
    d, m = g.scalar_rhs("burgers", torch.from_numpy(u0).cuda(), want_mask=True)
    d, m = d.cpu().numpy(), m.cpu().numpy()
    assert m[0] == m[n]  # periodic: faces 0 and n are one face
    assert 0 < np.unpackbits(m).mean() < 1  # both outcomes occur
    assert abs(d.sum()) <= 1e-12 * np.abs(d).sum()


def test_table_sinorder_linear_column_on_gpu(lib, net_file):
    """Sec. 4.2.1 Table "sinorder", optimal linear scheme: sin(pi x) advected
    once around [0, 2] (t = 2), periodic, SSP-RK3, on the GPU."""
    _, path = net_file
    for N, e_paper in golden("e2_sine_advection.txt"):
        N = int(N)
        if N > 240:
            continue
        cfl, tol = {10: (0.01, 1e-5), 20: (0.01, 1e-5), 40: (0.01, 2e-4),
                    60: (0.01, 5e-4), 240: (0.05, 0.02)}[N]
        g = lib.Neno6(ndim=1, nx=N, dx=2.0 / N, mask_mode="smooth", weights=path)
        x = (np.arange(N) + 0.5) * 2.0 / N
        u = torch.from_numpy(np.sin(math.pi * x)).cuda()
        g.scalar_solve("advection", u, cfl, 2.0)
        e = np.abs(u.cpu().numpy() - np.sin(math.pi * x)).max()
        assert abs(e - e_paper) <= tol * e_paper, (N, e, e_paper)


def test_scalar_arguments(lib, net_file):
    _, path = net_file
    g2 = lib.Neno6(ndim=2, nx=16, ny=16, weights=path)
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.Neno6Error) as e:
        g2.scalar_rhs("advection", u)
    assert e.value.code == -8
    gm = lib.Neno6(ndim=1, nx=16, precision="bf16", weights=path)
    with pytest.raises(lib.Neno6Error) as e:
        gm.scalar_solve("burgers", u, 0.4, 0.1)
    assert e.value.code == -8
