"""Pins of the oracle's classifier-loss gradient (Eq. (Crossentropy))."""
import numpy as np

from conftest import balanced_net

import synth


def _labels(n, seed):
    return np.random.default_rng(seed).integers(0, 16, n).astype(np.uint8)


def test_gradient_matches_central_differences():
    from oracle import mlp_grad
    from oracle.weights import Net
    net = balanced_net(61)
    X = synth.mlp_stencils(64, seed=62)
    y = _labels(64, 63)
    g = mlp_grad.grad(net, X, y)
    p0 = net.packed()
    rng = np.random.default_rng(64)
    for k in rng.choice(p0.size, 40, replace=False):
        h = 1e-6 * max(1.0, abs(p0[k]))
        def with_param(v):
            p = p0.copy()
            p[k] = v
            layers, o = [], 0
            for W, b in net.layers:
                nW = W.size
                layers.append((p[o:o + nW].reshape(W.shape), p[o + nW:o + nW + b.size]))
                o += nW + b.size
            return Net(layers)
        fd = (mlp_grad.loss(with_param(p0[k] + h), X, y) - mlp_grad.loss(with_param(p0[k] - h), X, y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-4, abs(g[k])), (k, fd, g[k])


def test_gradient_closed_form_for_a_constant_network():
    """All weights zero: z_k = b5_k for every sample, so dL/db5_k =
    (sigma(b5_k) - mean_s y_k) / S and every other gradient is 0; the loss is
    the mean of log(1 + e^b) - y b."""
    from oracle import mlp_grad
    from oracle.weights import Net
    widths = [6, 64, 32, 16, 8, 4]
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(widths[:-1], widths[1:])]
    b5 = np.array([0.3, -1.2, 2.0, 0.0])
    layers[-1] = (np.zeros((4, 8)), b5)
    net = Net(layers)
    X = synth.mlp_stencils(50, seed=1)
    y = _labels(50, 2)
    Y = ((y[:, None] >> np.arange(4)) & 1).astype(float)
    g = mlp_grad.grad(net, X, y)
    ref_b5 = (1 / (1 + np.exp(-b5)) - Y.mean(axis=0)) / 4
    assert np.allclose(g[-4:], ref_b5, rtol=1e-14, atol=1e-16)
    assert np.all(g[:-4] == 0.0)
    ref_loss = (np.log1p(np.exp(b5)) - Y * b5).mean()
    assert abs(mlp_grad.loss(net, X, y) - ref_loss) < 1e-14
