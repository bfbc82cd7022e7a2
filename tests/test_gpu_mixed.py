"""Tensor-core (tcgen05) classifier of the mixed-precision path.

Layout/exactness: a hand-built network whose weights, biases and inputs are
exactly representable in bf16 and fp16 must give the exact logits (every
product is exact and every partial sum is a small dyadic number, so FP32
accumulation is exact).  Numerics: a random network against a CPU emulation
that rounds to 16 bits at the same points (inputs, weights, hidden
activations) and accumulates in higher precision; the stencil decisions must
agree wherever the emulated logit is not within a small band of 0.
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


def round16(a, kind):
    a = np.asarray(a, dtype=np.float32)
    if kind == "fp16":
        return a.astype(np.float16).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def emulate(net, X, kind):
    """Layers 1-4 with 16-bit inputs and weights (tensor cores; in bf16 layer
    1's weights as two 16-bit terms, hi and the rounding of what hi leaves),
    layer 5 in FP32 (CUDA cores), biases at (at least) FP32 precision."""
    x = np.asarray(X, dtype=np.float32)
    m = np.maximum(1.0, np.abs(x).max(axis=1)).astype(np.float32)
    h = round16(x / m[:, None], kind)
    L = len(net.layers)
    for l, (W, b) in enumerate(net.layers):
        if l == 0 and kind == "bf16":
            W32 = np.asarray(W, dtype=np.float32)
            hi = round16(W32, kind)
            Wr = (hi + round16(W32 - hi, kind)).astype(np.float64)
        else:
            Wr = (round16(W, kind) if l < 4 else W.astype(np.float32)).astype(np.float64)
        acc = (h.astype(np.float64) @ Wr.T).astype(np.float32) + b.astype(np.float32)
        if l < L - 1:
            h = np.maximum(acc, 0.0)
            if l < 3:
                h = round16(h, kind)
        else:
            z = acc
    return z


def _hand_net():
    from test_oracle_pins import _hand_net as hn
    return hn()


@pytest.mark.parametrize("kind", ["bf16", "fp16"])
def test_tensor_core_mlp_exact_on_representable_network(lib, tmp_path, kind):
    net = _hand_net()
    path = tmp_path / "hand.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, precision=kind, weights=str(path))
    rng = np.random.default_rng(4)
    X = rng.integers(-8, 9, size=(300, 6)) / 8.0   # |x| <= 1: no normalisation, bf16-exact
    eta, z = g.classify(torch.from_numpy(X).cuda(), want_logits=True)
    z = z.cpu().numpy()
    ref = np.stack([X[:, 0] - X[:, 1], X[:, 2] - 0.25, -X[:, 3], X[:, 4] + X[:, 5] - 0.5], axis=1)
    assert np.array_equal(z, ref), np.abs(z - ref).max()
    bits = (ref > 0).astype(np.uint8) @ (1 << np.arange(4)).astype(np.uint8)
    assert np.array_equal(eta.cpu().numpy(), bits)


@pytest.mark.parametrize("kind", ["bf16", "fp16"])
def test_tensor_core_mlp_matches_16bit_emulation(lib, tmp_path, kind):
    net = balanced_net(31)
    path = tmp_path / "net.bin"
    net.save(path)
    g = lib.Neno6(ndim=1, nx=8, precision=kind, weights=str(path))
    X = synth.mlp_stencils(30000 + 77, seed=12)  # ragged last 128-row tile
    eta, z = g.classify(torch.from_numpy(X).cuda(), want_logits=True)
    eta, z = eta.cpu().numpy(), z.cpu().numpy()
    ze = emulate(net, X, kind)
    err = np.abs(z - ze)
    scale = 1.0 + np.abs(ze)
    assert np.quantile(err / scale, 0.999) < (2e-2 if kind == "bf16" else 3e-3)
    robust = np.abs(ze) > (0.1 if kind == "bf16" else 0.02)
    assert np.array_equal((z > 0)[robust], (ze > 0)[robust])
    bits = (z > 0).astype(np.uint8) @ (1 << np.arange(4)).astype(np.uint8)
    assert np.array_equal(eta, bits)


def test_mixed_classify_close_to_fp64(lib, tmp_path):
    """bf16 decisions agree with the FP64 path on all but a small fraction."""
    net = balanced_net(32)
    path = tmp_path / "net.bin"
    net.save(path)
    X = torch.from_numpy(synth.mlp_stencils(50000, seed=13)).cuda()
    e64 = lib.Neno6(ndim=1, nx=8, precision="fp64", weights=str(path)).classify(X).cpu().numpy()
    e16 = lib.Neno6(ndim=1, nx=8, precision="bf16", weights=str(path)).classify(X).cpu().numpy()
    flips = np.unpackbits(e64 ^ e16).sum() / (4 * len(e64))
    assert flips < 0.02, flips


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_width_study_emulation_matches_kernel(lib, kind):
    """The host emulation the width study uses (oracle/train/width_study.py)
    against the tensor-core kernel on the trained network: per-row logits
    agree to the emulation's own tolerance, and the logit errors against FP64
    have the same distribution on both sides."""
    from oracle.train import width_study as ws
    from oracle.weights import Net
    net = Net.load(lib.DEFAULT_WEIGHTS)
    g = lib.Neno6(ndim=1, nx=8, precision=kind, guard_tau=0.0)
    X = synth.mlp_stencils(1 << 16, seed=31)
    _, z = g.classify(torch.from_numpy(X).cuda(), want_logits=True)
    z = z.cpu().numpy()
    ze = ws.forward16(net, X, kind).astype(np.float64)
    z64 = ws.forward64(net, X)
    err = np.abs(z - ze) / (1.0 + np.abs(ze))
    assert np.quantile(err, 0.999) < (2e-2 if kind == "bf16" else 3e-3)
    q_kernel = np.quantile(np.abs(z - z64), [0.5, 0.99])
    q_emul = np.quantile(np.abs(ze - z64), [0.5, 0.99])
    np.testing.assert_allclose(q_kernel, q_emul, rtol=0.2)
