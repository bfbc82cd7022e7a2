"""Pins of the TENO6-opt labeler (oracle/train/teno6.py, Sec. 2.1-2.2), which
labels training family 9: its smoothness indicators against the published
closed forms (Jiang & Shu 1996 for three points; Fu et al. 2016 for the
four-point stencil of TENO6) and a brute-force quadrature of the Jiang-Shu
definition for the six-point one, the order of tau_6 (Eq. (taukTENO)) and the
cut-off's selection on jumps (Eq. (cut-off))."""
import numpy as np
import pytest

from oracle.train import teno6

RNG = np.random.default_rng(20220717)


def quad_beta(offsets, f):
    """Jiang-Shu indicator by brute force: the degree r-1 polynomial with the
    given cell averages (numpy solve) and Gauss-Legendre quadrature of its
    squared derivatives over the central cell (unit spacing)."""
    r = len(offsets)
    # cell average of x^l over [o - 1/2, o + 1/2]
    A = np.array([[((o + 0.5) ** (l + 1) - (o - 0.5) ** (l + 1)) / (l + 1) for l in range(r)]
                  for o in offsets])
    a = np.linalg.solve(A, f)
    xg, wg = np.polynomial.legendre.leggauss(12)
    xg, wg = xg / 2, wg / 2
    p = np.polynomial.Polynomial(a)
    return sum(float(np.sum(wg * p.deriv(l)(xg) ** 2)) for l in range(1, r))


def beta_of(offsets, f):
    B = teno6.beta_matrix(tuple(offsets))
    return float(f @ B @ f)


def test_three_point_indicators_are_jiang_shu():
    for _ in range(20):
        f = RNG.standard_normal(3)
        a, b, c = f
        np.testing.assert_allclose(beta_of((-2, -1, 0), f),
                                   13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2,
                                   rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(beta_of((-1, 0, 1), f),
                                   13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - c) ** 2,
                                   rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(beta_of((0, 1, 2), f),
                                   13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (3 * a - 4 * b + c) ** 2,
                                   rtol=1e-12, atol=1e-14)


def test_four_point_indicator_is_teno6():
    for _ in range(20):
        f0, f1, f2, f3 = f = RNG.standard_normal(4)
        ref = (1 / 36 * (-11 * f0 + 18 * f1 - 9 * f2 + 2 * f3) ** 2
               + 13 / 12 * (2 * f0 - 5 * f1 + 4 * f2 - f3) ** 2
               + 781 / 720 * (-f0 + 3 * f1 - 3 * f2 + f3) ** 2)
        np.testing.assert_allclose(beta_of((0, 1, 2, 3), f), ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("offsets", [(-1, 0, 1), (0, 1, 2, 3), (-2, -1, 0, 1, 2, 3)])
def test_indicators_match_quadrature(offsets):
    for _ in range(5):
        f = RNG.standard_normal(len(offsets))
        np.testing.assert_allclose(beta_of(offsets, f), quad_beta(offsets, f), rtol=1e-10)


def test_indicator_invariants():
    for offsets in [(-2, -1, 0), (-1, 0, 1), (0, 1, 2), (0, 1, 2, 3), teno6.FULL]:
        o = np.array(offsets, dtype=np.float64)
        B = teno6.beta_matrix(tuple(offsets))
        c = np.full(len(o), 3.7)
        assert abs(beta_of(offsets, c)) <= 1e-14 * 3.7**2 * np.abs(B).sum()  # constants: 0
        # the cell averages of p(x) = x are the cell centres; beta = int (p')^2 = 1
        np.testing.assert_allclose(beta_of(offsets, o), 1.0, rtol=1e-12)
        np.testing.assert_allclose(beta_of(offsets, o + 5.0), 1.0, rtol=1e-12)


def test_tau6_is_sixth_order():
    """tau_6 = O(dx^6) on smooth data: halving dx divides it by ~2^6."""
    j = np.arange(-2, 4)
    taus = []
    for h in (0.1, 0.05, 0.025):
        F = (np.cos(1.3 * (j + 0.5) * h) - np.cos(1.3 * (j - 0.5) * h)) / (1.3 * h) * -1
        b, b6 = teno6.smoothness(F[None, :])
        taus.append(abs(b6[0] - (b[0, 1] + b[0, 2] + 4 * b[0, 0]) / 6))
    orders = np.log2(np.array(taus[:-1]) / np.array(taus[1:]))
    assert np.all(orders > 5.7), orders


def test_selection_on_smooth_data_and_jumps():
    j = np.arange(-2, 4)
    smooth = np.sin(0.2 * j + 0.3)[None, :]
    assert teno6.select(smooth).tolist() == [[1, 1, 1, 1]]
    # a jump at face i+1/2 (between the third and fourth values): S_0, S_1 and
    # S_3 cross it, S_2 = {i-2, i-1, i} does not
    assert teno6.select(np.array([[0, 0, 0, 1, 1, 1.0]])).tolist() == [[0, 0, 1, 0]]
    # a jump at face i+3/2: S_1 and S_3 cross it
    assert teno6.select(np.array([[0, 0, 0, 0, 1, 1.0]])).tolist() == [[1, 0, 1, 0]]
    # a jump at face i-3/2: only S_2 crosses it
    assert teno6.select(np.array([[0, 1, 1, 1, 1, 1.0]])).tolist() == [[1, 1, 0, 1]]
    assert teno6.labels(np.array([[0, 0, 0, 1, 1, 1.0]])).tolist() == [[1, 1, 0, 1]]
    # constant sub-stencils, whose quadratic forms round to +-1e-15: never negative
    b, b6 = teno6.smoothness(np.array([[0, 1, 1, 1, 1, 1.0], [2, 2, 2, 2, 2, 2.0]]))
    assert (b >= 0).all() and (b6 >= 0).all()
    assert teno6.select(np.array([[2, 2, 2, 2, 2, 2.0]])).tolist() == [[1, 1, 1, 1]]
