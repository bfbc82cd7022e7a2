"""Pins of the oracle's mini-batch Adam training loop (oracle/mlp_train.py).

Adam as Table 2 names it (Kingma & Ba, Algorithm 1, default beta1 = 0.9,
beta2 = 0.999, epsilon = 1e-8).  The pins do not re-run the update formula:
iterates on f(theta) = theta^2 / 2 worked out by hand in 40-digit decimal
arithmetic, the first-step closed form (bias correction makes the first
update -lr g / (|g| + epsilon)), invariance under a positive rescaling of the
loss, and descent of the classifier loss.
"""
import numpy as np

from conftest import balanced_net

import synth


def test_adam_quadratic_worked_iterates():
    from oracle.mlp_train import adam_step
    # theta_0 = 1, g = theta, lr = 0.1: theta_1..theta_3 computed by hand
    expect = [0.9000000009999999900, 0.8004122297123373911, 0.7015862745044142142]
    th, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    for t, e in enumerate(expect, start=1):
        th, m, v = adam_step(th, th.copy(), m, v, t, 0.1)
        assert abs(th[0] - e) <= 1e-15, (t, th[0], e)


def test_first_step_closed_form_and_scale_invariance():
    from oracle.mlp_train import adam_step
    rng = np.random.default_rng(3)
    g = rng.standard_normal(1000) * 10.0 ** rng.uniform(-6, 2, 1000)
    th0 = rng.standard_normal(1000)
    th1, _, _ = adam_step(th0, g, np.zeros(1000), np.zeros(1000), 1, 1e-3)
    # |update| = lr |g| / (|g| + eps) < lr, in the direction of -g
    assert np.all(np.sign(th0 - th1) == np.sign(g))
    assert np.allclose(np.abs(th1 - th0), 1e-3 * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    # rescaling every gradient by c > 0 leaves the trajectory (nearly) unchanged
    a = (th0.copy(), np.zeros(1000), np.zeros(1000))
    b = (th0.copy(), np.zeros(1000), np.zeros(1000))
    for t in range(1, 6):
        gt = g * (1.0 + 0.1 * t)
        a = adam_step(a[0], gt, a[1], a[2], t, 1e-3)
        b = adam_step(b[0], 1e3 * gt, b[1], b[2], t, 1e-3)
    # where |g| >= 1e-4, epsilon = 1e-8 shifts each update by at most 1e-4 lr
    big = np.abs(g) >= 1e-4
    assert big.sum() > 500
    assert np.allclose(a[0][big], b[0][big], rtol=0, atol=5 * 1e-4 * 1e-3)


def test_training_lowers_the_loss_and_batches_cover_perm():
    from oracle import mlp_grad, mlp_train
    net = balanced_net(81)
    X = synth.mlp_stencils(700, seed=82)
    y = np.zeros(700, dtype=np.uint8)
    y[350:] = 0b1011
    perm = np.random.default_rng(83).permutation(700)
    p, m, v, losses = mlp_train.train(net, X, y, perm, 175, 1e-3)
    assert len(losses) == 4  # 700 / 175 batches
    assert mlp_grad.loss(mlp_train.unpack(net, p), X, y) < mlp_grad.loss(net, X, y)
    # a short last batch: 701 samples -> 5 steps, the last of one sample
    X2 = np.concatenate([X, X[:1]])
    y2 = np.concatenate([y, y[:1]])
    _, _, _, l2 = mlp_train.train(net, X2, y2, np.arange(701), 175, 1e-3)
    assert len(l2) == 5
