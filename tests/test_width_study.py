"""Host checks of the width study's 16-bit emulation (oracle/train/width_study.py):
its rounding against library conversions and hand-picked ties, its FP32 path
against the FP64 forward, and the FP64 forward against the oracle's classify."""
import numpy as np
import pytest
import torch

import oracle
from oracle.train import width_study as ws
from oracle.weights import Net


def test_round_bf16_matches_torch():
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    # exact ties: a bf16 value plus half an ulp, both parities of the kept bit
    base = torch.tensor(rng.standard_normal(1000), dtype=torch.bfloat16).float().numpy()
    ties = (base.view(np.uint32) | np.uint32(0x8000)).view(np.float32)
    a = np.concatenate([a, ties])
    ref = torch.from_numpy(a).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(ws.round_bf16(a), ref)


def test_round_fp16_ties_and_saturation():
    x = np.array([1 + 2.0**-11, 1 + 3 * 2.0**-11, -(1 + 2.0**-11), 7e4, -7e4, 65504.0, 2.0**-25],
                 dtype=np.float32)
    np.testing.assert_array_equal(
        ws.round_fp16(x),
        np.array([1.0, 1 + 2.0**-9, -1.0, 65504.0, -65504.0, 65504.0, 0.0], dtype=np.float32))


@pytest.mark.parametrize("widths", [(6, 64, 32, 16, 8, 4), (6, 32, 32, 32, 4)])
def test_forward_paths_agree(widths):
    net = Net.random(widths, seed=4)
    X = np.random.default_rng(5).uniform(-3, 3, (512, 6))
    z64 = ws.forward64(net, X)
    _, z_or = oracle.Oracle(ndim=1, nx=8, ny=1, net=net).classify(X)
    np.testing.assert_allclose(z64, z_or, rtol=0, atol=1e-12 * (1 + np.abs(z_or).max()))
    # without 16-bit rounding the emulation is the FP32 forward
    z32 = ws.forward16(net, X, None).astype(np.float64)
    scale = 1 + np.abs(z64).max()
    assert np.abs(z32 - z64).max() <= 1e-5 * scale
    # fp16 rounding moves the logits by more than FP32 does, bf16 by more still
    e16 = np.abs(ws.forward16(net, X, "fp16") - z64).max()
    eb16 = np.abs(ws.forward16(net, X, "bf16") - z64).max()
    assert np.abs(z32 - z64).max() < e16 < eb16


def test_flip_stats_counts():
    z64 = np.array([[1.0, -1.0, 0.3, -0.2]])
    z16 = np.array([[0.9, 0.1, -0.1, -3.0]])
    s = ws.flip_stats(z64, z16, 0.5)
    assert s["flips"] == 2 and s["flips_outside_band"] == 0 and s["rows_in_band"] == 1.0
    s = ws.flip_stats(z64, z16, 0.05)
    assert s["flips_outside_band"] == 2 and s["rows_in_band"] == 0.0


def test_bf16_layer1_split_keeps_smooth_stencils_out_of_the_band():
    """Why the bf16 tensor-core image carries layer 1's weights as two bf16
    terms: on smooth stencils (a mean plus a variation of 1e-3 per cell) the
    first layer's weights nearly cancel against the mean, and one bf16
    rounding of W1 leaves a residue larger than the variation.  With the
    split (the emulation `forward16` follows the kernel) the logits stay
    closer to FP64 and far fewer rows fall into the guard band or flip."""
    import paper_2207_08500_gb300 as p
    net = Net.load(p.DEFAULT_WEIGHTS)
    rng = np.random.default_rng(5)
    n = 20000
    X = rng.uniform(-1, 1, (n, 1)) + rng.uniform(-1e-3, 1e-3, (n, 1)) * np.arange(6)[None, :]
    z64 = ws.forward64(net, X)
    z_split = ws.forward16(net, X, "bf16")
    rnd = ws.ROUND["bf16"]
    a = rnd(ws.normalise32(X))  # the same evaluation with W1 rounded once
    for li, (W, b) in enumerate(net.layers):
        if li + 1 < len(net.layers):
            h = np.maximum(a @ rnd(W.astype(np.float32)).T + b.astype(np.float32), np.float32(0.0))
            a = rnd(h) if li + 2 < len(net.layers) else h
        else:
            a = a @ W.astype(np.float32).T + b.astype(np.float32)
    z_single = a
    err_split, err_single = np.abs(z_split - z64), np.abs(z_single - z64)
    band_split = (np.abs(z_split) < 1.0).any(axis=1).mean()
    band_single = (np.abs(z_single) < 1.0).any(axis=1).mean()
    flips_split = ((z_split > 0) != (z64 > 0)).sum()
    flips_single = ((z_single > 0) != (z64 > 0)).sum()
    assert np.median(err_single) > 1.5 * np.median(err_split)
    assert band_single > 3 * band_split
    assert flips_single > 5 * flips_split
