"""Training data on the device (neno6_datagen) against the oracle's recipe
(oracle/train/datagen.py from_uniforms) on the same uniform draws, and the
on-device retraining loop it feeds (neno6_datagen -> neno6_mlp_train)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


def _draws(n, seed):
    u = np.random.default_rng(seed).random((n, 9))
    # the extreme draws of every column
    u[0] = 0.0
    u[1] = np.nextafter(1.0, 0.0)
    return u


def test_datagen_matches_oracle_recipe(lib):
    from oracle.train import datagen
    u = _draws(20011, 41)
    g = lib.Neno6(ndim=1, nx=8)
    X, lab, fam = g.datagen(torch.from_numpy(u).cuda())
    X, lab, fam = X.cpu().numpy(), lab.cpu().numpy(), fam.cpu().numpy()
    assert g.status() == 0
    Xo, labo, famo = datagen.from_uniforms(u)
    assert np.array_equal(fam, famo)
    # grids, positions, parameters and singular points are exact binary64 on
    # both sides: the geometric labels (families 1-8) agree bit for bit
    geo = fam <= 8
    assert np.array_equal(lab[geo], labo[geo])
    # family 9 (TENO6-opt labels): only a last-bit difference of sin or of the
    # indicator sums can move a stencil across the cut-off
    m9 = fam == 9
    mism = int((lab[m9] != labo[m9]).sum())
    print("family-9 label mismatches: %d of %d" % (mism, m9.sum()))
    assert mism <= max(2, m9.sum() // 1000)
    # values: CUDA's sin / cos / exp / log against the host's, last bits
    assert np.abs(X - Xo).max() <= 1e-13


def test_datagen_bad_draw_sets_status(lib):
    g = lib.Neno6(ndim=1, nx=8)
    u = torch.from_numpy(_draws(300, 42)).cuda()
    u[7, 4] = 1.0
    u[9, 0] = -0.25
    X, lab, fam = g.datagen(u)
    assert g.status() & 8
    assert g.status() == 0
    assert fam[7].item() == 0 and fam[9].item() == 0 and torch.count_nonzero(X[7]).item() == 0
    assert (fam[10:] > 0).all()


def test_retraining_loop_on_device_data(lib):
    """Algorithm 1 data made on the device feeds the Adam loop (batch 175,
    learning rate 1e-3): the mean batch loss falls from epoch 1 to epoch 4."""
    g = lib.Neno6(ndim=1, nx=8)
    n = 1 << 15
    X, lab, _ = g.datagen(torch.from_numpy(np.random.default_rng(43).random((n, 9))).cuda())
    rng = np.random.default_rng(44)
    params = []
    widths = (6, 64, 32, 16, 8, 4)
    for a, b in zip(widths[:-1], widths[1:]):
        params.append(rng.standard_normal((b, a)) * np.sqrt(2.0 / a))
        params.append(np.zeros(b))
    p = torch.from_numpy(np.concatenate([w.ravel() for w in params]).astype(np.float32)).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    steps = (n + 174) // 175
    losses, t0 = [], 0
    for ep in range(4):
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        ls = g.mlp_train(X, lab, perm, p, m, v, t0, 1e-3)
        t0 += steps
        losses.append(ls.item() / steps)
    print("mean batch loss per epoch:", losses)
    assert g.status() == 0
    assert losses[-1] < 0.8 * losses[0]
