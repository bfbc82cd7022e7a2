"""Classifier training-loss gradient on the GPU (neno6_mlp_bwd) against the
FP64 oracle gradient (oracle/mlp_grad.py, itself pinned by central
differences); FP32 arithmetic, so the comparison is at FP32 tolerance."""
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


def _labels(X, seed):
    """Plausible labels: steps discard the stencils they cross (eta = 1),
    sinusoids keep them, with a little seeded noise."""
    n = X.shape[0]
    y = np.zeros(n, dtype=np.uint8)
    y[n // 2:] = 0b1011
    flip = np.random.default_rng(seed).integers(0, 16, n).astype(np.uint8)
    mask = np.random.default_rng(seed + 1).random(n) < 0.1
    y[mask] ^= flip[mask]
    return y


@pytest.mark.parametrize("n", [1, 127, 3001, 1 << 20])
def test_mlp_bwd_matches_oracle(lib, tmp_path, n):
    from oracle import mlp_grad
    net = balanced_net(71)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, weights=str(path))
    X = synth.mlp_stencils(max(n, 2), seed=72)[:n]
    y = _labels(X, 73)
    grad, loss = g.mlp_bwd(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    grad, loss = grad.cpu().numpy().astype(np.float64), float(loss.item())
    ref = mlp_grad.grad(net, X, y)
    ref_loss = mlp_grad.loss(net, X, y)
    scale = np.abs(ref).max()
    assert np.abs(grad - ref).max() <= 2e-4 * scale, np.abs(grad - ref).max() / scale
    assert abs(loss - ref_loss) <= 2e-5 * abs(ref_loss)


def test_mlp_bwd_deterministic_and_descends(lib, tmp_path):
    from oracle import mlp_grad
    from oracle.weights import Net
    net = balanced_net(74)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, weights=str(path))
    X = synth.mlp_stencils(20000, seed=75)
    y = _labels(X, 76)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g1, l1 = g.mlp_bwd(Xd, yd)
    g2, l2 = g.mlp_bwd(Xd, yd)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)
    # one gradient-descent step on the packed parameters lowers the loss
    p = net.packed() - 0.5 * g1.cpu().numpy().astype(np.float64)
    layers, o = [], 0
    for W, b in net.layers:
        layers.append((p[o:o + W.size].reshape(W.shape), p[o + W.size:o + W.size + b.size]))
        o += W.size + b.size
    assert mlp_grad.loss(Net(layers), X, y) < mlp_grad.loss(net, X, y)


# ------------------------------------------------- tensor cores (mixed handles)
# The tensor-core gradient rounds the weights, the activations and the deltas
# to 16 bits and accumulates in FP32: against the FP64 gradient its error is
# a multiple of the 16-bit unit roundoff (fp16 2^-11, bf16 2^-8) relative to
# the gradient's norm, not of FP32's.
TC_TOL = {"fp16": 4e-3, "bf16": 4e-2}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [1, 127, 3001, 1 << 20])
def test_mlp_bwd_tensor_cores_against_oracle(lib, tmp_path, prec, n):
    from oracle import mlp_grad
    net = balanced_net(71)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, precision=prec, weights=str(path))
    X = synth.mlp_stencils(max(n, 2), seed=72)[:n]
    y = _labels(X, 73)
    grad, loss = g.mlp_bwd(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    assert g.status() == 0
    grad, loss = grad.cpu().numpy().astype(np.float64), float(loss.item())
    ref = mlp_grad.grad(net, X, y)
    ref_loss = mlp_grad.loss(net, X, y)
    err = np.linalg.norm(grad - ref) / np.linalg.norm(ref)
    print("%s n=%d: gradient rel L2 error %.2e, loss rel error %.2e"
          % (prec, n, err, abs(loss - ref_loss) / abs(ref_loss)))
    assert err <= TC_TOL[prec]
    assert abs(loss - ref_loss) <= TC_TOL[prec] * abs(ref_loss)
    # every layer's weights and biases are in the gradient (none left at 0)
    offs = [0, 384, 448, 2496, 2528, 3040, 3056, 3184, 3192, 3224, 3228]
    for a, b in zip(offs[:-1], offs[1:]):
        seg = np.linalg.norm(grad[a:b] - ref[a:b]) / max(np.linalg.norm(ref[a:b]), 1e-30)
        assert seg <= 5 * TC_TOL[prec], (a, seg)


def test_mlp_bwd_tensor_cores_deterministic_and_descends(lib, tmp_path):
    from oracle import mlp_grad
    from oracle.weights import Net
    net = balanced_net(74)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, precision="fp16", weights=str(path))
    X = synth.mlp_stencils(20000, seed=75)
    y = _labels(X, 76)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g1, l1 = g.mlp_bwd(Xd, yd)
    g2, l2 = g.mlp_bwd(Xd, yd)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)
    p = net.packed() - 0.5 * g1.cpu().numpy().astype(np.float64)
    layers, o = [], 0
    for W, b in net.layers:
        layers.append((p[o:o + W.size].reshape(W.shape), p[o + W.size:o + W.size + b.size]))
        o += W.size + b.size
    assert mlp_grad.loss(Net(layers), X, y) < mlp_grad.loss(net, X, y)
