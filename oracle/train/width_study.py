"""Classifier width study: the paper's 6-64-32-16-8-4 network against a
6-32-32-32-4 network trained with the same data and recipe (Sec. 3.2-3.3,
Table 2), on classification quality and on sensitivity to 16-bit arithmetic.

Test infrastructure (oracle side): nothing here runs on the GPU, and the CUDA
library never imports it.

For each weights file the script reports
  * multiply-adds per classifier call;
  * held-out F1 (discarded stencils as positives) and accuracy on fresh
    samples of the Algorithm 1 / Table 9 generator (another seed than the
    training data), from the FP64 oracle's classify;
  * the logit error and decision flips of a 16-bit evaluation of the network,
    emulated on the host (`forward16`), on the same held-out samples and on
    the seeded sine / step stencils of `synth.mlp_stencils`.

The 16-bit evaluation follows the arithmetic of the library's tensor-core
classifier: the normalised input (Eq. for X, FP32, divided by max(|x|, 1)) and
every weight of a tensor-core layer are rounded to 16 bits (round to nearest
even), except that in bf16 the first layer's weights are carried as two
16-bit terms (hi, then the rounding of what hi leaves), products are summed in
FP32 and the bias is added in FP32; a hidden
activation is ReLU'd and rounded to 16 bits when the next layer is also a
tensor-core layer.  Every layer but the last runs on the tensor cores; the
last layer (8 -> 4, or 32 -> 4) takes the FP32 activation and FP32 weights on
the CUDA cores.  The summation order inside a tensor-core product is the
hardware's; the emulation's differs, which moves results by FP32 rounding
(~1e-7 relative), far below the 16-bit rounding (2^-11 fp16, 2^-8 bf16).

    python -m oracle.train.width_study weights/neno6_mlp_6x64x32x16x8x4.bin \
        weights/neno6_mlp_6x32x32x32x4.bin
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle.train import datagen  # noqa: E402
from oracle.weights import Net  # noqa: E402


def round_bf16(a):
    """float32 array rounded to the nearest bfloat16 (ties to even), returned
    as float32.  Finite inputs only."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def round_fp16(a):
    """float32 array rounded to the nearest binary16 (ties to even), returned
    as float32; magnitudes past the largest finite half saturate to it, as a
    satfinite conversion does."""
    a = np.clip(np.asarray(a, dtype=np.float32), -65504.0, 65504.0)
    return a.astype(np.float16).astype(np.float32)


ROUND = {"fp16": round_fp16, "bf16": round_bf16}


def normalise32(X):
    """FP32 normalisation of raw stencils: x_j / max(1, |x_0|, ..., |x_5|)."""
    X = np.asarray(X, dtype=np.float32)
    m = np.maximum(np.float32(1.0), np.abs(X).max(axis=1, keepdims=True))
    return X / m


def forward64(net, X):
    """FP64 logits of raw stencils X [n, 6] (normalise, ReLU hidden layers)."""
    X = np.asarray(X, dtype=np.float64)
    a = X / np.maximum(1.0, np.abs(X).max(axis=1, keepdims=True))
    for li, (W, b) in enumerate(net.layers):
        a = a @ W.T + b
        if li + 1 < len(net.layers):
            a = np.maximum(a, 0.0)
    return a


def forward16(net, X, prec):
    """Emulated 16-bit evaluation (module docstring) of raw stencils X [n, 6];
    prec None keeps every operand in FP32 (the same code path without the
    16-bit rounding)."""
    rnd = ROUND[prec] if prec is not None else (lambda v: np.asarray(v, dtype=np.float32))
    L = len(net.layers)
    a = rnd(normalise32(X))
    for li, (W, b) in enumerate(net.layers):
        b32 = b.astype(np.float32)
        if li + 1 < L:
            W32 = W.astype(np.float32)
            Wr = rnd(W32)
            if li == 0 and prec == "bf16":
                Wr = Wr + rnd(W32 - Wr)  # hi + lo: exact in FP32
            z = a @ Wr.T + b32
            h = np.maximum(z, np.float32(0.0))
            a = rnd(h) if li + 2 < L else h
        else:
            a = a @ W.astype(np.float32).T + b32
    return a


def flip_stats(z64, z16, tau):
    """Decision flips of the 16-bit logits against FP64 (discard iff z > 0),
    the fraction of rows a guard band |z16| < tau sends back to FP32, and the
    flips the band does not catch."""
    flip = (z64 > 0) != (z16 > 0)
    row_in_band = (np.abs(z16) < tau).any(axis=1)
    missed = flip & (np.abs(z16) >= tau)
    return {"flip_rate": float(flip.mean()), "flips": int(flip.sum()),
            "tau": tau, "rows_in_band": float(row_in_band.mean()),
            "flips_outside_band": int(missed.sum())}


def err_quantiles(z64, z16):
    e = np.abs(z16.astype(np.float64) - z64).ravel()
    return {"median": float(np.quantile(e, 0.5)), "q999": float(np.quantile(e, 0.999)),
            "max": float(e.max())}


GUARD_TAU = {"fp16": 0.5, "bf16": 1.0}


def study(path, n_heldout=30000, n_stencils=1 << 20):
    net = Net.load(path)
    out = {"widths": list(net.widths), "sha256": net.sha256(),
           "macs_per_call": int(sum(W.size for W, _ in net.layers))}
    X, y, _ = datagen.generate(n_heldout, seed=777)
    o = oracle.Oracle(ndim=1, nx=8, ny=1, net=net)
    eta, z_or = o.classify(X)
    pred = ((eta[:, None] >> np.arange(4)) & 1).astype(bool)
    yt = np.asarray(y).astype(bool)
    tp = int((pred & yt).sum())
    fp = int((pred & ~yt).sum())
    fn = int((~pred & yt).sum())
    out["heldout_F1_discarded"] = 2 * tp / (2 * tp + fp + fn)
    out["heldout_accuracy"] = float((pred == yt).mean())
    z64 = forward64(net, X)
    # the numpy forward and the oracle's classify compute the same logits
    out["forward64_vs_oracle_max_abs"] = float(np.abs(z64 - z_or).max())
    S = synth.mlp_stencils(n_stencils, seed=31)
    zs64 = forward64(net, S)
    out["median_abs_logit_heldout"] = float(np.median(np.abs(z64)))
    for prec in ("fp16", "bf16"):
        r = {}
        for name, XX, zz in (("heldout", X, z64), ("sine_step", S, zs64)):
            z16 = forward16(net, XX, prec)
            r[name] = {"logit_err": err_quantiles(zz, z16),
                       "tau0": flip_stats(zz, z16, 0.0),
                       "guard": flip_stats(zz, z16, GUARD_TAU[prec])}
        out[prec] = r
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("weights", nargs="+")
    ap.add_argument("--heldout", type=int, default=30000)
    ap.add_argument("--stencils", type=int, default=1 << 20)
    a = ap.parse_args()
    for p in a.weights:
        print(json.dumps(study(p, a.heldout, a.stencils)), flush=True)


if __name__ == "__main__":
    main()
