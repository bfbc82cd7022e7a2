"""The width study's 6-32-32-32-4 classifier on the GPU (neno6_classify only):
the FP64 form bit-exact with the oracle, the tensor-core forms against the
host emulation of their 16-bit arithmetic, and every other entry point
refusing the network."""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
NARROW = os.path.join(os.path.dirname(HERE), "weights", "neno6_mlp_6x32x32x32x4.bin")


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def _stencils():
    X = synth.mlp_stencils(20011, seed=51)
    return np.concatenate([X, X[:2000] * 1e-3, X[:2000] * 37.0])


@pytest.mark.parametrize("trained", [True, False])
def test_narrow_fp64_classify_bit_exact(lib, oracle_mod, tmp_path, trained):
    if trained:
        net, path = oracle_mod.Net.load(NARROW), NARROW
    else:
        net = oracle_mod.Net.random(widths=(6, 32, 32, 32, 4), seed=9)
        path = str(tmp_path / "n.bin")
        net.save(path)
    X = _stencils()
    g = lib.Neno6(ndim=1, nx=8, precision="fp64", weights=path)
    eta, z = g.classify(torch.from_numpy(X).cuda(), want_logits=True)
    eta_o, z_o = oracle_mod.Oracle(ndim=1, nx=8, ny=1, net=net).classify(X)
    assert np.array_equal(eta.cpu().numpy(), eta_o)
    assert np.array_equal(z.cpu().numpy(), z_o)


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_narrow_tensor_core_classify_matches_emulation(lib, oracle_mod, kind):
    from oracle.train import width_study as ws
    net = oracle_mod.Net.load(NARROW)
    X = _stencils()
    g = lib.Neno6(ndim=1, nx=8, precision=kind, weights=NARROW)
    eta, z = g.classify(torch.from_numpy(X).cuda(), want_logits=True)
    eta, z = eta.cpu().numpy(), z.cpu().numpy()
    assert g.status() == 0
    ze = ws.forward16(net, X, kind).astype(np.float64)
    z64 = ws.forward64(net, X)
    err = np.abs(z - ze) / (1.0 + np.abs(ze))
    assert np.quantile(err, 0.999) < (2e-2 if kind == "bf16" else 3e-3)
    q_kernel = np.quantile(np.abs(z - z64), [0.5, 0.99])
    q_emul = np.quantile(np.abs(ze - z64), [0.5, 0.99])
    np.testing.assert_allclose(q_kernel, q_emul, rtol=0.2)
    bits = (z > 0).astype(np.uint8) @ (1 << np.arange(4)).astype(np.uint8)
    assert np.array_equal(eta, bits)


def test_narrow_network_serves_classify_only(lib):
    g = lib.Neno6(ndim=2, nx=16, ny=16, precision="fp64", weights=NARROW)
    U = torch.from_numpy(synth.quadrants_2d(16, 16)).cuda()
    with pytest.raises(lib.Neno6Error) as e:
        g.rhs(U)
    assert e.value.code == -8
    with pytest.raises(lib.Neno6Error):
        g.step(U, 0.4)
