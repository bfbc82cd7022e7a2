"""Training / validation data for the NENO6 classifier (Algorithm 1, Table 9).

Training infrastructure (oracle side).  For each sample:
  1. a grid N in {50, 100, 200} drawn with probabilities 40/40/20 % (Sec. 3.2)
     on [-1, 1], cell centres x_j = -1 + (j + 1/2) dx, dx = 2/N;
  2. a function of Table 9 (families 1-9, equally likely) with its seeded
     parameters, and an interface x_{i+1/2};
  3. the six point values f_{i-2..i+3}, normalised by Eq. (normalizainput);
  4. labels eta_0..eta_3 (1 = stencil S_k crossed by a discontinuity):
       families 1-3 (smooth)            eta = 0 (Table 9);
       families 4-8 (kinks, jumps)      eta_k = 1 iff a singular point of the
                                        function lies strictly between the
                                        outermost cell centres of S_k;
       family 9 (near-grid-frequency)   TENO6-opt selection (teno6.py), the
                                        labeler Sec. 3.2 names for data whose
                                        regularity is not known in closed form.

Readings where Table 9 is under-specified: a_k ~
U[0.1, 2] in family 2; the "0.6" of N[0, 0.6] in family 5 is a variance;
family 6 joins (x-a1)^k1 and (x-a2)^k2 (integer k in 2..8) continuously at a
kink x_k ~ U[-0.6, 0.6]; family 8 places the jump at the sampled interface
(data "only collected at x_{i+1/2} = x_0") for half of its samples and at
another face inside the stencil for the other half, standing in for the
temporally evolved discontinuous solutions that Algorithm 1 collects, which are
not generated; family 9 uses N_f ~ U[N/8, N/2].

Sign reading.  Table 9 draws the levels of family 8 from U[0, 2], so every
training jump lies between two non-negative values; the classifier's Euler
inputs, the LLF-split characteristic fluxes, change sign across shocks, and
a network trained on the printed ranges keeps stencils across jumps from
-1 to 1 (a Mach 5.5 oblique shock then goes non-physical within ~36 steps in
the FP64 oracle).  Here the family-8 levels are drawn from U[-2, 2] and every
sample is negated with probability 1/2 (a function and its negative have the
same singular points and the same TENO6 selection, so the labels are kept).
"""
import math

import numpy as np

from . import teno6

SPAN = {0: (-1, 1), 1: (0, 2), 2: (-2, 0), 3: (0, 3)}  # cell offsets of S_k's outermost cells


def _geometric(x_i, dx, sing, valid):
    """eta_k = 1 iff a singular point lies strictly inside S_k's span.
    x_i [n], sing [n, m] singular abscissae (valid mask [n, m])."""
    n = x_i.shape[0]
    eta = np.zeros((n, 4), dtype=np.uint8)
    for k, (lo, hi) in SPAN.items():
        a = (x_i + lo * dx)[:, None]
        b = (x_i + hi * dx)[:, None]
        inside = (sing > a) & (sing < b) & valid
        eta[:, k] = inside.any(axis=1)
    return eta


def generate(n, seed=20220717):
    rng = np.random.default_rng(seed)
    N = rng.choice(np.array([50, 100, 200]), p=[0.4, 0.4, 0.2], size=n)
    fam = rng.integers(1, 10, size=n)
    dx = 2.0 / N
    i = rng.integers(2, N - 3)  # stencil cells i-2..i+3 inside the grid
    xi = -1.0 + (i + 0.5) * dx
    off = np.arange(-2, 4)
    X = xi[:, None] + off[None, :] * dx[:, None]
    F = np.zeros((n, 6))
    eta = np.zeros((n, 4), dtype=np.uint8)
    u = lambda a, b: rng.uniform(a, b, size=n)
    sing = np.full((n, 64), np.nan)

    # 1: k x
    k = u(-5, 5)
    m = fam == 1
    F[m] = (k[:, None] * X)[m]
    # 2: a sin(k x)
    a, k = u(0.1, 2.0), u(1, 5)
    m = fam == 2
    F[m] = (a[:, None] * np.sin(k[:, None] * X))[m]
    # 3: exp(a1 (x - a2)^2)
    a1, a2 = u(-1, 1), u(-1, 1)
    m = fam == 3
    F[m] = np.exp(a1[:, None] * (X - a2[:, None]) ** 2)[m]
    # 4: triangle wave (r/P)(P - |(x mod 2P) - P|), kinks at multiples of P
    r, P = u(1, 3), u(2, 8) * dx
    m = fam == 4
    F[m] = ((r / P)[:, None] * (P[:, None] - np.abs(np.mod(X, 2 * P[:, None]) - P[:, None])))[m]
    kmin = np.floor((X[:, 0] - dx) / P) - 1
    cand = (kmin[:, None] + np.arange(64)[None, :]) * P[:, None]
    sing[m] = cand[m]
    # 5: max(0, b1 (x - x0)) + c, kink at x0
    b1, x0, c = rng.normal(0.0, np.sqrt(0.6), size=n), u(-0.6, 0.6), u(0, 1)
    m = fam == 5
    F[m] = (np.maximum(0.0, b1[:, None] * (X - x0[:, None])) + c[:, None])[m]
    sing[m, 0] = x0[m]
    # 6: (x-a1)^k1 | (x-a2)^k2 joined continuously at a kink xk
    k1, k2 = rng.integers(2, 9, size=n), rng.integers(2, 9, size=n)
    a1, a2, xk = u(0, 2), u(0, 2), u(-0.6, 0.6)
    m = fam == 6
    left = (X - a1[:, None]) ** k1[:, None]
    right = (X - a2[:, None]) ** k2[:, None] + ((xk - a1) ** k1 - (xk - a2) ** k2)[:, None]
    F[m] = np.where(X <= xk[:, None], left, right)[m]
    sing[m, 0] = xk[m]
    # 7: sqrt(max(0, 1 - alpha^2 (x-a)^2)), edges at a +- 1/alpha
    al, a = u(0.05, 2), u(0, 2)
    m = fam == 7
    F[m] = np.sqrt(np.maximum(0.0, 1.0 - al[:, None] ** 2 * (X - a[:, None]) ** 2))[m]
    sing[m, 0] = (a - 1.0 / al)[m]
    sing[m, 1] = (a + 1.0 / al)[m]
    # 8: step x_l / x_r; half with the jump at the interface x_{i+1/2}
    # (Table 9), half at another face inside the stencil (stand-in for the
    # advected discontinuities Algorithm 1 collects)
    xl, xr = u(-2, 2), u(-2, 2)
    m = fam == 8
    shift = np.where(rng.uniform(size=n) < 0.5, 0, rng.integers(-2, 3, size=n))
    x_jump = xi + (0.5 + shift) * dx
    F[m] = np.where(X <= x_jump[:, None], xl[:, None], xr[:, None])[m]
    sing[m, 0] = x_jump[m]
    # 9: a1 sin(N_f pi (x - x0)), N_f ~ U[N/8, N/2]
    a1, x0, Nf = u(0, 2), u(0, 2), u(0.125, 0.5) * N
    m = fam == 9
    F[m] = (a1[:, None] * np.sin(Nf[:, None] * np.pi * (X - x0[:, None])))[m]

    geo = (fam >= 4) & (fam <= 8)
    valid = ~np.isnan(sing)
    eta[geo] = _geometric(xi[geo], dx[geo], np.nan_to_num(sing[geo]), valid[geo])
    m9 = fam == 9
    eta[m9] = teno6.labels(F[m9])
    # sign symmetry (see the module docstring)
    neg = rng.uniform(size=n) < 0.5
    F[neg] = -F[neg]
    # Eq. (normalizainput)
    Xn = F / np.maximum(np.abs(F).max(axis=1, keepdims=True), 1.0)
    return Xn, eta, fam


# Columns of a uniform draw matrix u [n][DRAWS] (values in [0, 1)) for
# from_uniforms: grid, family, interface position, five family parameters,
# sign.
DRAWS = 9


def _ipow(b, k):
    r = b
    for _ in range(k - 1):
        r = r * b
    return r


def from_uniforms(u):
    """The recipe of `generate` (Table 9, Algorithm 1, the readings above) as
    a plain function of caller-given uniform draws u [n][DRAWS], one sample
    per row, in IEEE binary64 without fused operations: the form a device
    generator can reproduce from the same draws.  (`generate`, which wrote
    the frozen weights, draws from numpy's generator in its own order and
    maps some parameters differently, e.g. the normal of family 5; the two
    produce the same distribution, not the same samples.)

    Returns (Xn [n][6] float64 normalised by Eq. (normalizainput),
    labels [n] uint8 with eta_k in bit k, fam [n] uint8)."""
    u = np.asarray(u, dtype=np.float64)
    assert u.ndim == 2 and u.shape[1] == DRAWS
    n = u.shape[0]
    F = np.zeros((n, 6))
    eta = np.zeros((n, 4), dtype=np.uint8)
    fam = np.zeros(n, dtype=np.uint8)
    two_pi = 2.0 * math.pi
    for r in range(n):
        q = [float(v) for v in u[r]]
        N = 50 if q[0] < 0.4 else (100 if q[0] < 0.8 else 200)
        f = 1 + min(int(9.0 * q[1]), 8)
        i = 2 + min(int((N - 5) * q[2]), N - 6)
        p = q[3:8]
        dx = 2.0 / N
        xi = -1.0 + (i + 0.5) * dx
        X = [xi + (j - 2) * dx for j in range(6)]
        sing = []       # singular points (families 4-8 except 4)
        period = None   # family 4: kinks at every multiple of P
        if f == 1:
            k = -5.0 + 10.0 * p[0]
            v = [k * x for x in X]
        elif f == 2:
            a, k = 0.1 + 1.9 * p[0], 1.0 + 4.0 * p[1]
            v = [a * math.sin(k * x) for x in X]
        elif f == 3:
            a1, a2 = -1.0 + 2.0 * p[0], -1.0 + 2.0 * p[1]
            v = [math.exp(a1 * ((x - a2) * (x - a2))) for x in X]
        elif f == 4:
            rr, P = 1.0 + 2.0 * p[0], (2.0 + 6.0 * p[1]) * dx
            v = []
            for x in X:
                md = x - (2.0 * P) * math.floor(x / (2.0 * P))
                v.append((rr / P) * (P - abs(md - P)))
            period = P
        elif f == 5:
            b1 = math.sqrt(0.6) * (math.sqrt(-2.0 * math.log(1.0 - p[0])) * math.cos(two_pi * p[1]))
            x0, c = -0.6 + 1.2 * p[2], p[3]
            v = [max(0.0, b1 * (x - x0)) + c for x in X]
            sing = [x0]
        elif f == 6:
            k1, k2 = 2 + min(int(7.0 * p[0]), 6), 2 + min(int(7.0 * p[1]), 6)
            a1, a2, xk = 2.0 * p[2], 2.0 * p[3], -0.6 + 1.2 * p[4]
            jump = _ipow(xk - a1, k1) - _ipow(xk - a2, k2)
            v = [_ipow(x - a1, k1) if x <= xk else _ipow(x - a2, k2) + jump for x in X]
            sing = [xk]
        elif f == 7:
            al, a = 0.05 + 1.95 * p[0], 2.0 * p[1]
            v = [math.sqrt(max(0.0, 1.0 - (al * al) * ((x - a) * (x - a)))) for x in X]
            sing = [a - 1.0 / al, a + 1.0 / al]
        elif f == 8:
            xl, xr = -2.0 + 4.0 * p[0], -2.0 + 4.0 * p[1]
            shift = 0 if p[2] < 0.5 else -2 + min(int(5.0 * p[3]), 4)
            xj = xi + (0.5 + shift) * dx
            v = [xl if x <= xj else xr for x in X]
            sing = [xj]
        else:
            a1, x0, Nf = 2.0 * p[0], 2.0 * p[1], (0.125 + 0.375 * p[2]) * N
            v = [a1 * math.sin((Nf * math.pi) * (x - x0)) for x in X]
        F[r] = v
        fam[r] = f
        if 4 <= f <= 8:
            for k, (lo_o, hi_o) in SPAN.items():
                lo, hi = xi + lo_o * dx, xi + hi_o * dx
                if period is not None:  # is some multiple m P strictly inside?
                    hit = False
                    m = math.floor(lo / period)
                    while m * period < hi:
                        hit = hit or m * period > lo
                        m += 1
                else:
                    hit = any(lo < s_ < hi for s_ in sing)
                eta[r, k] = 1 if hit else 0
    m9 = fam == 9
    if m9.any():
        eta[m9] = teno6.labels(F[m9])
    neg = u[:, 8] < 0.5
    F[neg] = -F[neg]
    Xn = F / np.maximum(np.abs(F).max(axis=1, keepdims=True), 1.0)
    labels = (eta.astype(np.uint8) << np.arange(4, dtype=np.uint8)).sum(axis=1).astype(np.uint8)
    return Xn, labels, fam


def dataset(n_total=709000, seed=20220717):
    """The paper's 709 000 samples; the first 70 % train, the rest validate."""
    X, y, fam = generate(n_total, seed)
    n_tr = int(0.7 * n_total)
    return (X[:n_tr], y[:n_tr]), (X[n_tr:], y[n_tr:]), fam
