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
    """tau_6 = O(dx^6) on smooth data (Eq. (taukTENO)): halving dx divides it
    by ~2^6, while the indicators themselves are O(dx^2)."""
    j = np.arange(-2, 4)
    taus, b0 = [], []
    for h in (0.1, 0.05, 0.025):
        F = (np.cos(1.3 * (j + 0.5) * h) - np.cos(1.3 * (j - 0.5) * h)) / (1.3 * h) * -1
        b, b6 = teno6.smoothness(F[None, :])
        taus.append(teno6.tau6(b, b6)[0])
        b0.append(b[0, 0])
    orders = np.log2(np.array(taus[:-1]) / np.array(taus[1:]))
    assert np.all(orders > 5.7), orders
    assert np.all(np.abs(np.log2(np.array(b0[:-1]) / np.array(b0[1:])) - 2) < 0.1)


def test_cut_off_constants_and_chi():
    """Eq. (measureTENO) and (cut-off) with the printed C = 1, q = 6,
    eps = 1e-40, C_T = 1e-6: chi sums to 1, does not depend on the scale of
    the data, and the selection is exactly chi >= 1e-6."""
    assert (teno6.C, teno6.Q, teno6.EPS, teno6.CT) == (1.0, 6, 1e-40, 1e-6)
    rng = np.random.default_rng(5)
    j = np.arange(-2, 4)
    # sines near the grid frequency, some with a jump: chi spans many decades
    F = np.sin(rng.uniform(0.2, 2.8, (20000, 1)) * j + rng.uniform(0, 6.3, (20000, 1)))
    F[::3] += rng.uniform(-1, 1, (len(F[::3]), 1)) * (j >= rng.integers(-1, 4, (len(F[::3]), 1)))
    c = teno6.chi(F)
    np.testing.assert_allclose(c.sum(axis=1), 1.0, rtol=1e-12)
    np.testing.assert_allclose(teno6.chi(7.5 * F), c, rtol=1e-9, atol=1e-300)
    assert np.array_equal(teno6.select(F), (c >= 1e-6).astype(np.uint8))
    near = (c > 1e-7) & (c < 1e-5)
    assert near.sum() > 20  # the threshold is exercised on both sides


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


def test_chi_exponent_is_q(monkeypatch):
    """gamma_k is a q-th power (Eq. (measureTENO)): the log ratio of two
    stencils' chi is proportional to q, and q is the printed 6."""
    rng = np.random.default_rng(6)
    j = np.arange(-2, 4)
    F = np.sin(rng.uniform(0.5, 2.5, (200, 1)) * j + rng.uniform(0, 6.3, (200, 1)))
    c6 = teno6.chi(F)
    monkeypatch.setattr(teno6, "Q", 3)
    c3 = teno6.chi(F)
    l6 = np.log(c6[:, 0] / c6[:, 1])
    l3 = np.log(c3[:, 0] / c3[:, 1])
    ok = np.abs(l3) > 1e-3
    np.testing.assert_allclose(l6[ok], 2.0 * l3[ok], rtol=1e-9)
