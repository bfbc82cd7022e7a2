"""Pins of the oracle's TENO6-opt mask mode (Sec. 2.1-2.2: Eqs.
(measureTENO), (taukTENO), (normalize), (cut-off)) used as the mask source of
the Euler right-hand side, the paper's comparison scheme.

The C++ selection is checked against the independent Python labeler of
oracle/train/teno6.py (itself pinned by closed forms in
tests/test_oracle_teno6.py), against the TENO6-opt column the paper prints in
Table "Convergencesmooth" (golden tests/golden/e1_cos_convergence_teno6.txt),
and the right-hand side built on it against what the selection implies: only
the sub-stencil on the far side of a jump kept at the jump, discards on
smooth data confined to a vanishing set of faces, convergence on Sod's
problem.  CPU only.
"""
import numpy as np

import synth
from oracle.train import teno6


def _eta_bits(labels):
    return (labels * (1 << np.arange(4))).sum(axis=1)


def test_teno_selection_equals_python_labeler(oracle_mod):
    o = oracle_mod.Oracle(ndim=1, nx=8, mask_mode="teno6")
    rng = np.random.default_rng(4)
    X = np.concatenate([synth.mlp_stencils(6000, seed=9), rng.normal(size=(3000, 6)),
                        rng.normal(size=(1000, 6)) * 1e-6 + 5.0])
    got = np.array([o.reconstruct(x, mask_mode="teno6")[1] for x in X])
    ref = _eta_bits(teno6.labels(X))
    chi = teno6.chi(X)
    # the two sides round differently; a decision may differ only where chi
    # sits on the cut-off to rounding
    near = np.any(np.abs(chi / teno6.CT - 1.0) < 1e-9, axis=1)
    assert np.all((got == ref) | near)
    assert (got == ref).mean() > 0.999
    assert 0.02 < np.unpackbits(got.astype(np.uint8)).mean() < 0.5  # both outcomes


def test_teno_at_a_jump_keeps_the_upwind_side_only(oracle_mod):
    """A step between cells i and i+1 crosses S0 = {i-1,i,i+1},
    S1 = {i,i+1,i+2} and S3 = {i..i+3}; only S2 = {i-2,i-1,i} is kept."""
    o = oracle_mod.Oracle(ndim=1, nx=8, mask_mode="teno6")
    for lo, hi in [(0.0, 1.0), (-2.0, 3.0), (1.0, 1.5), (0.3, -0.2)]:
        s = np.array([lo, lo, lo, hi, hi, hi])
        v, eta = o.reconstruct(s, mask_mode="teno6")
        assert eta == 0b1011, (lo, hi, eta)
        # S2 alone reproduces the constant left state (its coefficients sum
        # to 1; they are not exact in binary64)
        assert abs(v - lo) <= 1e-15 * max(1.0, abs(lo))
    # a smooth polynomial keeps all four
    x = np.arange(-2, 4) * 0.05
    assert o.reconstruct(1.0 + x + 0.3 * x ** 2, mask_mode="teno6")[1] == 0


def test_table_convergencesmooth_teno6_column(oracle_mod):
    """Sec. 4.1 Table "Convergencesmooth", TENO6-opt column: on cos x at
    x = -0.5 the selection keeps every stencil on both sides, so the error
    is the linear scheme's, and matches the printed digits."""
    import math
    from conftest import golden
    o = oracle_mod.Oracle(ndim=1, nx=8, mask_mode="teno6")
    for N, e_paper in golden("e1_cos_convergence_teno6.txt"):
        dx, xi = 2.0 / N, -0.5
        sp = np.array([math.cos(xi + (k - 2) * dx) for k in range(6)])
        sm = np.array([math.cos(xi + (k - 3) * dx) for k in range(6)])
        fp, ep = o.reconstruct(sp, mask_mode="teno6")
        fm, em = o.reconstruct(sm, mask_mode="teno6")
        assert ep == 0 and em == 0
        e = abs((fp - fm) / dx - (-math.sin(xi)))
        tol = 2e-5 if N <= 160 else 1e-3
        assert abs(e - e_paper) <= tol * e_paper, (N, e, e_paper)


def test_teno_discards_on_smooth_data_vanish_with_resolution(oracle_mod):
    """On smooth data the selection discards stencils only near critical
    points of the split fluxes, a set whose share of the faces shrinks like
    1/N: the fraction of discarded decisions at least halves per doubling."""
    fr = []
    for n in (48, 96, 192):
        U = synth.smooth_2d(n, n, seed=2)
        _, m = oracle_mod.Oracle(ndim=2, nx=n, ny=n, mask_mode="teno6").rhs(U, want_mask=True)
        fr.append(np.unpackbits(m).mean())
    assert fr[1] < 0.5 * fr[0] and fr[2] < 0.5 * fr[1] and fr[2] < 0.01, fr


def test_teno_rhs_discards_at_shocks_and_converges_on_sod(oracle_mod):
    errs = []
    from test_oracle_pins import _sod_exact
    for N in (100, 200):
        x = (np.arange(N) + 0.5) / N
        rho = np.where(x < 0.5, 1.0, 0.125)
        p = np.where(x < 0.5, 1.0, 0.1)
        U = synth.prim_to_cons(rho, 0.0, 0.0, p, ndim=1).reshape(3, 1, N)
        o = oracle_mod.Oracle(ndim=1, nx=N, bc=("transmissive", "transmissive"), mask_mode="teno6")
        t = 0.0
        while t < 0.2:
            U, t, _ = o.step(U, 0.5, t, 0.2)
        _, m = o.rhs(U, want_mask=True)
        assert np.count_nonzero(m) > 0  # stencils across the waves are discarded
        errs.append(np.abs(U[0, 0] - _sod_exact(x, 0.2)).mean())
    # sharper than the first-order scheme's (< 0.03 at N = 100) and converging
    assert errs[0] < 0.015 and errs[1] < errs[0] * 0.8, errs
