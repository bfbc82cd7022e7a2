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
