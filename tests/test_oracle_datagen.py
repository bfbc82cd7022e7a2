"""Pins of the training-data generator (oracle/train/datagen.py; Algorithm 1,
Table 9 and Eq. (normalizainput)): the geometric labels against a
cell-by-cell brute force, and the labels of the generated samples against
what their function families fix (a jump family's kept sub-stencils are
constant and its discarded ones are not; a kink family's kept sub-stencils
lie on one line; smooth families keep everything)."""
import numpy as np

from oracle.train import datagen

# positions (0..5 = cells i-2..i+3) of each candidate sub-stencil S_k
CELLS = {0: (1, 2, 3), 1: (2, 3, 4), 2: (0, 1, 2), 3: (2, 3, 4, 5)}


def brute_geometric(x_i, dx, sing):
    eta = np.zeros(4, dtype=np.uint8)
    centres = x_i + (np.arange(6) - 2) * dx
    for k, cells in CELLS.items():
        lo, hi = centres[cells[0]], centres[cells[-1]]
        eta[k] = any(lo < s < hi for s in sing)
    return eta


def test_geometric_labels_brute_force():
    rng = np.random.default_rng(3)
    n = 400
    x_i = rng.uniform(-1, 1, n)
    dx = rng.choice([0.01, 0.02, 0.04], n)
    sing = x_i[:, None] + rng.uniform(-3.5, 4.5, (n, 3)) * dx[:, None]
    valid = rng.uniform(size=(n, 3)) < 0.7
    eta = datagen._geometric(x_i, dx, sing, valid)
    for r in range(n):
        assert eta[r].tolist() == brute_geometric(x_i[r], dx[r], sing[r][valid[r]]).tolist()
    # a singular point at the face x_{i+1/2}: S_0, S_1, S_3 cross it, S_2 does not
    e = datagen._geometric(np.array([0.0]), np.array([0.1]), np.array([[0.05]]), np.array([[True]]))
    assert e.tolist() == [[1, 1, 0, 1]]


def _gen(n=20000, seed=11):
    return datagen.generate(n, seed=seed)


def test_shapes_normalisation_and_smooth_families():
    X, eta, fam = _gen()
    assert X.shape == (20000, 6) and eta.shape == (20000, 4) and set(np.unique(fam)) == set(range(1, 10))
    assert np.abs(X).max() <= 1.0
    # Eq. (normalizainput): rows whose largest |value| reached 1 or more now peak at exactly 1
    big = np.abs(X).max(axis=1) == 1.0
    assert big.mean() > 0.3
    assert (eta[fam <= 3] == 0).all()


def test_jump_family_labels_match_its_values():
    X, eta, fam = _gen()
    m = np.flatnonzero(fam == 8)
    assert len(m) > 1000
    for r in m:
        levels = np.unique(X[r])
        assert len(levels) <= 2
        for k, cells in CELLS.items():
            constant = np.ptp(X[r, list(cells)]) == 0.0
            assert constant == (eta[r, k] == 0), (X[r], eta[r])
    # every sample's stencil holds the jump (at the interface or another face)
    assert (eta[m].sum(axis=1) > 0).all()


def test_kink_family_kept_stencils_are_linear():
    X, eta, fam = _gen()
    for r in np.flatnonzero(fam == 5):
        scale = max(np.abs(X[r]).max(), 1e-300)
        for k, cells in CELLS.items():
            if eta[r, k] == 0:
                v = X[r, list(cells)]
                d2 = v[:-2] - 2 * v[1:-1] + v[2:]
                assert np.abs(d2).max() <= 1e-12 * scale, (X[r], eta[r], k)


def test_sign_symmetry_and_split():
    X, eta, fam = _gen()
    # family 3 (a Gaussian, positive everywhere) is negated for about half the samples
    m = fam == 3
    neg = (X[m] < 0).all(axis=1)
    pos = (X[m] > 0).all(axis=1)
    assert (neg | pos).all()
    n3 = m.sum()
    assert abs(neg.sum() - n3 / 2) < 5 * np.sqrt(n3 / 4)
    (Xt, yt), (Xv, yv), _ = datagen.dataset(n_total=1000, seed=5)
    assert len(Xt) == 700 and len(Xv) == 300


def _from_uniforms(n=20000, seed=12):
    u = np.random.default_rng(seed).random((n, datagen.DRAWS))
    X, labels, fam = datagen.from_uniforms(u)
    eta = ((labels[:, None] >> np.arange(4)) & 1).astype(np.uint8)
    return u, X, eta, fam


def test_from_uniforms_labels_match_values():
    u, X, eta, fam = _from_uniforms()
    assert set(np.unique(fam)) == set(range(1, 10)) and np.abs(X).max() <= 1.0
    assert (eta[fam <= 3] == 0).all()
    for r in np.flatnonzero(fam == 8):
        for k, cells in CELLS.items():
            assert (np.ptp(X[r, list(cells)]) == 0.0) == (eta[r, k] == 0)
    # families 4 (triangle wave) and 5 (ramp): piecewise linear, so a
    # sub-stencil is kept iff its values lie on one line (up to rounding)
    for f in (4, 5):
        for r in np.flatnonzero(fam == f):
            scale = np.abs(X[r]).max()
            for k, cells in CELLS.items():
                v = X[r, list(cells)]
                d2 = np.abs(v[:-2] - 2 * v[1:-1] + v[2:]).max()
                if eta[r, k] == 0:
                    assert d2 <= 1e-12 * scale
                elif f == 4:
                    assert d2 > 1e-9 * scale, (X[r], eta[r], k)


def test_from_uniforms_same_distribution_as_generate():
    _, _, eta, fam = _from_uniforms(30000, seed=13)
    _, y, fam_g = datagen.generate(30000, seed=14)
    for f in range(1, 10):
        assert abs((fam == f).mean() - 1 / 9) < 0.01
        a, b = eta[fam == f].mean(axis=0), y[fam_g == f].mean(axis=0)
        assert np.abs(a - b).max() < 0.03, (f, a, b)


def test_from_uniforms_sign_rule():
    """The reading of Table 9's signs: a sample is negated iff its sign draw
    is below 1/2 (family 3, a positive Gaussian, shows the sign)."""
    u, X, eta, fam = _from_uniforms(6000, seed=15)
    m = fam == 3
    assert ((X[m] < 0).all(axis=1) == (u[m, 8] < 0.5)).all()
    assert ((X[m] > 0).all(axis=1) == (u[m, 8] >= 0.5)).all()


def test_from_uniforms_edges_of_the_draws():
    # the smallest and largest draws map inside every range
    u = np.array([[0.0] * datagen.DRAWS, [np.nextafter(1.0, 0.0)] * datagen.DRAWS])
    X, labels, fam = datagen.from_uniforms(u)
    assert fam.tolist() == [1, 9] and np.isfinite(X).all()
