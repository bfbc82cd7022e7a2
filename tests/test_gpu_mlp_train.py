"""Classifier training on the GPU (neno6_mlp_train) against the FP64 oracle
loop (oracle/mlp_train.py: Adam of Kingma & Ba, Algorithm 1, on the gradient
of oracle/mlp_grad.py, both pinned on the CPU).

FP32 on the GPU against FP64: the per-step losses agree to FP32 tolerance;
parameters agree to a small fraction of the learning rate except where a
gradient is within FP32 rounding of zero, where Adam's normalisation by
sqrt(v) may turn the rounding into an update of up to lr (bounded below).
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


def _data(n, seed):
    X = synth.mlp_stencils(n, seed=seed)
    y = np.zeros(n, dtype=np.uint8)
    y[n // 2:] = 0b1011
    rng = np.random.default_rng(seed + 1)
    noise = rng.random(n) < 0.1
    y[noise] ^= rng.integers(0, 16, n).astype(np.uint8)[noise]
    return X, y


def _gpu_state(net):
    p = torch.from_numpy(net.packed().astype(np.float32)).cuda()
    return p, torch.zeros_like(p), torch.zeros_like(p)


@pytest.mark.parametrize("n_perm,batch", [(175 * 30, 175), (1000, 192), (333, 1), (700 + 42, 175)])
def test_mlp_train_matches_oracle_adam(lib, tmp_path, n_perm, batch):
    from oracle import mlp_train
    net = balanced_net(91)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, weights=str(path))
    X, y = _data(4000, 92)
    perm = np.random.default_rng(93).integers(0, 4000, n_perm).astype(np.int32)
    lr = 1e-4
    p, m, v = _gpu_state(net)
    loss = g.mlp_train(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(perm).cuda(),
                       p, m, v, 0, lr, batch=batch)
    assert g.status() == 0
    ref, _, _, losses = mlp_train.train(net, X, y, perm, batch, lr)
    steps = len(losses)
    assert abs(loss.item() - sum(losses)) <= 1e-5 * sum(losses)
    d = np.abs(p.cpu().numpy().astype(np.float64) - ref)
    print("steps %d: |dp| quantiles 0.99 %.2e, 0.999 %.2e, max %.2e (lr %.0e)"
          % (steps, np.quantile(d, 0.99), np.quantile(d, 0.999), d.max(), lr))
    assert np.quantile(d, 0.99) <= 1e-2 * lr
    assert d.max() <= 2.0 * lr * steps


def test_mlp_train_continues_across_calls_and_is_deterministic(lib, tmp_path):
    net = balanced_net(94)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, weights=str(path))
    X, y = _data(3000, 95)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    perm = torch.from_numpy(np.random.default_rng(96).permutation(3000).astype(np.int32)).cuda()
    a = _gpu_state(net)
    la = g.mlp_train(Xd, yd, perm, *a, 0, 1e-3)
    b = _gpu_state(net)
    lb = g.mlp_train(Xd, yd, perm, *b, 0, 1e-3)
    assert all(torch.equal(s, t) for s, t in zip(a, b)) and torch.equal(la, lb)
    # 1750 + 1250 samples in two calls = the same 3000 in one (t0 carries the
    # step count into the bias correction); 1750 = 10 whole batches
    c = _gpu_state(net)
    l1 = g.mlp_train(Xd, yd, perm[:1750], *c, 0, 1e-3)
    l2 = g.mlp_train(Xd, yd, perm[1750:], *c, 10, 1e-3)
    assert torch.allclose(c[0], a[0], rtol=0, atol=1e-6)
    assert abs((l1 + l2).item() - la.item()) <= 1e-6 * la.item()
    # the loss went down over the two passes
    l3 = g.mlp_train(Xd, yd, perm, *c, 18, 1e-3)
    assert l3.item() < la.item()


def test_mlp_train_arguments(lib, tmp_path):
    net = balanced_net(97)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, weights=str(path))
    X, y = _data(100, 98)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    perm = torch.arange(100, dtype=torch.int32, device="cuda")
    for bad in (0, 193):
        with pytest.raises(lib.Neno6Error) as e:
            g.mlp_train(Xd, yd, perm, *_gpu_state(net), 0, 1e-3, batch=bad)
        assert e.value.code == -2
    # an index outside [0, n) is skipped and reported in the status word
    p, m, v = _gpu_state(net)
    bad_perm = perm.clone()
    bad_perm[7] = 100
    g.mlp_train(Xd, yd, bad_perm, p, m, v, 0, 1e-3, batch=50)
    assert g.status() & 8
    assert g.status() == 0
