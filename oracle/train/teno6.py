"""TENO6-opt stencil selection, used to label training data.

Test/training infrastructure (oracle side).  Sec. 2.1-2.2 of the paper:

  gamma_k = (C + tau_6 / (beta_k + eps))^q,  C = 1, q = 6, eps = 1e-40
                                                   (Eq. (measureTENO))
  tau_6   = | beta_6 - (beta_1 + beta_2 + 4 beta_0) / 6 |   (Eq. (taukTENO))
  chi_k   = gamma_k / sum_k gamma_k                          (Eq. (normalize))
  delta_k = [chi_k >= C_T],  C_T = 1e-6                     (Eq. (cut-off))

The paper does not print beta_k or beta_6; it says they are defined like the
WENO (Jiang-Shu) indicators.  They are derived here symbolically from that
definition: p is the degree r-1 polynomial whose cell averages over the
stencil's cells equal the point values (Eq. (definitionEq)), and

  beta = sum_{l=1}^{r-1} dx^{2l-1} int_{x_{i-1/2}}^{x_{i+1/2}} (d^l p / dx^l)^2 dx,

which with dx = 1 is a quadratic form in the stencil values.  beta_6 uses the
full six-point stencil i-2..i+3.
"""
from functools import lru_cache

import numpy as np

STENCILS = {0: (-1, 0, 1), 1: (0, 1, 2), 2: (-2, -1, 0), 3: (0, 1, 2, 3)}
FULL = (-2, -1, 0, 1, 2, 3)
C, Q, EPS, CT = 1.0, 6, 1e-40, 1e-6


@lru_cache(maxsize=None)
def beta_matrix(offsets):
    """Symmetric matrix B with beta = f^T B f for the stencil `offsets`
    (exact rational derivation, returned as float64)."""
    import sympy as sp
    r = len(offsets)
    x = sp.Symbol("x")
    f = sp.symbols("f0:%d" % r)
    a = sp.symbols("a0:%d" % r)
    p = sum(a[l] * x ** l for l in range(r))
    half = sp.Rational(1, 2)
    eqs = [sp.integrate(p, (x, o - half, o + half)) - f[j] for j, o in enumerate(offsets)]
    sol = sp.solve(eqs, a, dict=True)[0]
    p = sp.expand(p.subs(sol))
    beta = sum(sp.integrate(sp.diff(p, x, l) ** 2, (x, -half, half)) for l in range(1, r))
    beta = sp.expand(beta)
    B = np.zeros((r, r))
    for i in range(r):
        for j in range(r):
            c = beta.coeff(f[i], 1).coeff(f[j], 1) if i != j else beta.coeff(f[i], 2)
            B[i, j] = float(c) / (2.0 if i != j else 1.0)
    return B


def _beta(F, offsets):
    B = beta_matrix(tuple(offsets))
    cols = [o + 2 for o in offsets]  # position in the six-point stencil
    # beta does not change when a constant is added to every value (the
    # derivatives of p do not), so the first value is subtracted first: a
    # constant sub-stencil then gives exactly 0, as in exact arithmetic,
    # instead of rounding noise that eps = 1e-40 would magnify
    V = F[:, cols] - F[:, cols[:1]]
    return np.einsum("ni,ij,nj->n", V, B, V)


def smoothness(F):
    """beta_0..beta_3 and beta_6 of stencils F [n, 6] (values at i-2..i+3).
    Each is an integral of squared derivatives, so never negative; a
    quadratic form that rounds below 0 is taken as 0."""
    F = np.asarray(F, dtype=np.float64)
    b = np.stack([_beta(F, STENCILS[k]) for k in range(4)], axis=1)
    b6 = _beta(F, FULL)
    return np.maximum(b, 0.0), np.maximum(b6, 0.0)


def tau6(b, b6):
    """Eq. (taukTENO): tau_6 = |beta_6 - (beta_1 + beta_2 + 4 beta_0) / 6|."""
    return np.abs(b6 - (b[:, 1] + b[:, 2] + 4.0 * b[:, 0]) / 6.0)


def chi(F):
    """chi_k of Eq. (normalize) for stencils F [n, 6]: gamma_k of Eq.
    (measureTENO) normalised to sum 1 (in the log domain, a stable softmax)."""
    b, b6 = smoothness(F)
    tau = tau6(b, b6)
    lg = Q * np.log(C + tau[:, None] / (b + EPS))
    lg -= lg.max(axis=1, keepdims=True)
    g = np.exp(lg)
    return g / g.sum(axis=1, keepdims=True)


def select(F):
    """TENO6-opt delta_k (1 = smooth, kept) for stencils F [n, 6]: the
    cut-off of Eq. (cut-off)."""
    return (chi(F) >= CT).astype(np.uint8)


def labels(F):
    """eta_k = 1 - delta_k (1 = stencil crossed by a discontinuity)."""
    return (1 - select(F)).astype(np.uint8)
