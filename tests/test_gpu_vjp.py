"""Frozen-mask adjoint (neno6_rhs_vjp) against the oracle and finite
differences.

The oracle side is forward mode (dual numbers through the same scheme with
the mask frozen), so on tiny grids its Jacobian columns J e_k assemble the
exact J^T lambda; on larger grids the dot-product identity <lambda, J v> =
<J^T lambda, v> is checked; central differences of the GPU's own frozen-mask
right-hand side give an independent check of the derivative itself.
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
def net_file(tmp_path_factory):
    net = balanced_net(51)
    path = tmp_path_factory.mktemp("w") / "net.bin"
    net.save(path)
    return net, str(path)


def _state(ndim, nx, ny, seed):
    if ndim == 2:
        return synth.noisy(synth.quadrants_2d(nx, ny, seed=seed), seed=seed + 1, rel=1e-3)
    return synth.noisy(synth.riemann_1d(nx, seed=seed), seed=seed + 1, rel=1e-2)


@pytest.mark.parametrize("ndim,nx,ny,bc", [(2, 7, 5, ("periodic", "periodic")),
                                           (2, 6, 7, ("transmissive", "periodic")),
                                           (1, 11, 1, ("transmissive", "transmissive")),
                                           (1, 4, 1, ("periodic", "periodic"))])
def test_vjp_equals_oracle_jacobian_transpose(lib, oracle_mod, net_file, ndim, nx, ny, bc):
    net, path = net_file
    g = lib.Neno6(ndim=ndim, nx=nx, ny=ny, bc=bc, weights=path)
    o = oracle_mod.Oracle(ndim=ndim, nx=nx, ny=ny, bc=bc, net=net)
    U = _state(ndim, nx, ny, 3)
    _, mask = o.rhs(U, want_mask=True)
    lam = synth.normal(U.shape, seed=4)
    grad = g.rhs_vjp(torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    ref = np.zeros(U.size)
    for k in range(U.size):
        e = np.zeros(U.size)
        e[k] = 1.0
        _, col = o.jvp(U, e.reshape(U.shape), mask)
        ref[k] = (lam * col).sum()
    ref = ref.reshape(U.shape)
    assert np.abs(grad - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(grad - ref).max()


@pytest.mark.parametrize("ndim,nx,ny,bc", [(2, 40, 36, ("periodic", "periodic")),
                                           (2, 33, 20, ("transmissive", "transmissive")),
                                           (1, 400, 1, ("transmissive", "transmissive"))])
def test_vjp_dot_product_identity(lib, oracle_mod, net_file, ndim, nx, ny, bc):
    net, path = net_file
    g = lib.Neno6(ndim=ndim, nx=nx, ny=ny, bc=bc, weights=path)
    o = oracle_mod.Oracle(ndim=ndim, nx=nx, ny=ny, bc=bc, net=net)
    U = _state(ndim, nx, ny, 5)
    Ud = torch.from_numpy(U).cuda()
    _, mask_g = g.rhs(Ud, want_mask=True)
    _, mask_o = o.rhs(U, want_mask=True)
    assert np.array_equal(mask_g.cpu().numpy(), mask_o)
    for s in range(3):
        lam = synth.normal(U.shape, seed=10 + s)
        v = synth.normal(U.shape, seed=20 + s)
        grad = g.rhs_vjp(Ud, torch.from_numpy(lam).cuda(), mask=mask_g).cpu().numpy()
        _, jv = o.jvp(U, v, mask_o)
        a, b = (lam * jv).sum(), (grad * v).sum()
        assert abs(a - b) <= 1e-11 * (np.abs(lam * jv).sum()), (a, b)


def test_vjp_central_differences(lib, net_file):
    """Directional derivative from the GPU's own frozen-mask RHS, step 1e-6,
    on smooth data (no ties in the alpha maximum)."""
    _, path = net_file
    n = 64
    g = lib.Neno6(ndim=2, nx=n, ny=n, weights=path)
    U = torch.from_numpy(synth.smooth_2d(n, n, seed=7)).cuda()
    _, mask = g.rhs(U, want_mask=True)
    lam = torch.from_numpy(synth.normal(U.shape, seed=8)).cuda()
    grad = g.rhs_vjp(U, lam, mask=mask)
    h = 1e-6
    for s in range(4):
        v = torch.from_numpy(synth.normal(U.shape, seed=30 + s)).cuda()
        fp = g.rhs(U + h * v, mask_in=mask)
        fm = g.rhs(U - h * v, mask_in=mask)
        fd = ((fp - fm) / (2 * h) * lam).sum().item()
        an = (grad * v).sum().item()
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (fd, an)


def test_autograd_function(lib, net_file):
    _, path = net_file
    g = lib.Neno6(ndim=2, nx=24, ny=20, weights=path)
    U = torch.from_numpy(synth.smooth_2d(24, 20, seed=2)).cuda().requires_grad_(True)
    lam = torch.from_numpy(synth.normal((4, 20, 24), seed=3)).cuda()
    out = lib.rhs(U, g)
    (out * lam).sum().backward()
    ref = g.rhs_vjp(U.detach(), lam)
    assert torch.equal(U.grad, ref)
    assert torch.equal(out.detach(), g.rhs(U.detach()))


def _untied_quadrants(n):
    """The four-quadrant state with u, v and p also modulated by 1e-2 smooth
    seeded modes (a sum of an x wave and a y wave, so the modulation varies
    along both axes almost everywhere): piecewise-constant velocities would
    give exact ties in the LLF maximum |lambda| over a stencil, where the
    frozen-argmax derivative is one-sided and central differences average the
    two sides."""
    U = synth.quadrants_2d(n, n)
    rho, u, v = U[0], U[1] / U[0], U[2] / U[0]
    p = 0.4 * (U[3] - 0.5 * rho * (u * u + v * v))
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    rng = np.random.default_rng(77)
    mods = []
    for _ in range(3):
        kx, ky = rng.integers(3, 10, 2)
        ph = rng.uniform(0, 2 * np.pi, 2)
        mods.append(1 + 5e-3 * (np.sin(2 * np.pi * kx * X + ph[0]) + np.sin(2 * np.pi * ky * Y + ph[1])))
    u, v, p = u * mods[0], v * mods[1], p * mods[2]
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)]))


def _near_tie_cells(U, delta):
    """Cells inside the stencil of some face whose LLF maximum over its six
    cells is within delta of the runner-up, for any field, either direction
    (periodic grid).  Perturbations kept off these cells cannot change an
    argmax the adjoint holds frozen."""
    rho, u, v = U[0], U[1] / U[0], U[2] / U[0]
    p = 0.4 * (U[3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(1.4 * p / rho)
    out = np.zeros(rho.shape, dtype=bool)
    for axis, un in ((1, u), (0, v)):
        for lam in (un - c, un, un + c):
            L = np.abs(lam)
            st = np.sort(np.stack([np.roll(L, 3 - k, axis=axis) for k in range(6)]), axis=0)
            tie = (st[5] - st[4]) < delta
            for k in range(6):
                out |= np.roll(tie, k - 3, axis=axis)
    return out


def test_vjp_full_size_against_oracle_jvp(lib, oracle_mod):
    """The differentiation workload's state itself (1024^2 four quadrants, the
    trained network): for 48 sampled (cell, field) unit vectors e, <lambda, J e>
    from the oracle's forward-mode J e at the 13 cells e can reach equals
    (J^T lambda)[cell, field] from the GPU.  Exact derivatives on both sides
    (mask and alpha argmax frozen alike), so ties in the LLF maximum do not
    matter here."""
    from oracle.weights import Net
    n = 1024
    U = synth.quadrants_2d(n, n)
    g = lib.Neno6(ndim=2, nx=n, ny=n)
    Ud = torch.from_numpy(U).cuda()
    _, mask = g.rhs(Ud, want_mask=True)
    lam = synth.normal(U.shape, seed=12)
    grad = g.rhs_vjp(Ud, torch.from_numpy(lam).cuda(), mask=mask).cpu().numpy()
    o = oracle_mod.Oracle(ndim=2, nx=n, ny=n, net=Net.load(lib.DEFAULT_WEIGHTS))
    mask_h = mask.cpu().numpy()
    rng = np.random.default_rng(3)
    V = np.zeros_like(U)
    for _ in range(48):
        s, fld = int(rng.integers(0, n * n)), int(rng.integers(0, 4))
        i, j = s % n, s // n
        V[fld, j, i] = 1.0
        cells = sorted({j * n + (i + d) % n for d in range(-3, 4)} | {((j + d) % n) * n + i for d in range(-3, 4)})
        jv = o.jvp_cells(U, V, mask_h, np.array(cells))
        terms = np.array([lam[:, c // n, c % n] * jv[r] for r, c in enumerate(cells)])
        V[fld, j, i] = 0.0
        lhs, rhs = terms.sum(), grad[fld, j, i]
        assert abs(lhs - rhs) <= 1e-10 * np.abs(terms).sum(), (s, fld, lhs, rhs)


def test_vjp_central_differences_full_size(lib):
    """Central differences (step 1e-6) of the frozen-mask FP64 RHS at full
    size, 1024^2, 64 seeded directions v ~ N(0,1) normalised to unit norm,
    lambda ~ N(0,1), the trained network.  The four-quadrant state has
    piecewise-constant velocities, i.e. exact ties in the LLF maximum where
    the frozen-argmax derivative is one-sided, so velocities and pressure are
    modulated (1e-2) and the directions vanish on the stencils of the faces
    whose maximum is within 1e-7 of the runner-up (a step moves any |lambda|
    by at most ~3e-8).  What remains is the rounding and O(h^2) error of the
    differences, up to ~2e-6 relative here: the bound is 1e-5."""
    n = 1024
    Uh = _untied_quadrants(n)
    excl = _near_tie_cells(Uh, 1e-7)
    assert excl.mean() < 0.1, excl.mean()
    keep = torch.from_numpy(~excl).cuda()
    g = lib.Neno6(ndim=2, nx=n, ny=n)
    U = torch.from_numpy(Uh).cuda()
    _, mask = g.rhs(U, want_mask=True)
    lam = torch.from_numpy(synth.normal(tuple(U.shape), seed=12)).cuda()
    grad = g.rhs_vjp(U, lam, mask=mask)
    h = 1e-6
    worst = 0.0
    for s in range(64):
        v = torch.from_numpy(synth.normal(tuple(U.shape), seed=100 + s)).cuda() * keep
        v /= v.norm()
        fp = g.rhs(U + h * v, mask_in=mask)
        fm = g.rhs(U - h * v, mask_in=mask)
        fd = float(((fp - fm) * lam).sum()) / (2 * h)
        an = float((grad * v).sum())
        worst = max(worst, abs(fd - an) / abs(an))
    assert g.status() == 0
    print("full-size central differences: worst relative difference %.2e over 64 directions" % worst)
    assert worst <= 1e-5, worst
