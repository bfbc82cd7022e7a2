"""Classifier training loss and its gradient, FP64 (oracle side).

Test infrastructure.  Eq. (Crossentropy): the mean binary cross entropy over
the n samples of a batch and the S = 4 sigmoid outputs (Eq.
(sigmoidfunction)) of the 6-64-32-16-8-4 ReLU network (Sec. 3.1), inputs
normalised by Eq. (normalizainput).  Written out layer by layer with numpy
matrix products; the backward pass is the chain rule in the reverse order.
Pinned in tests/test_oracle_mlp_grad.py by central differences of loss() and
by a closed form.
"""
import numpy as np


def _forward(net, X):
    X = np.asarray(X, dtype=np.float64)
    x = X / np.maximum(np.abs(X).max(axis=1, keepdims=True), 1.0)
    acts, pre = [x], []
    h = x
    L = len(net.layers)
    for l, (W, b) in enumerate(net.layers):
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if l < L - 1 else z
        acts.append(h)
    return acts, pre


def loss(net, X, labels):
    """Mean BCE: -1/(n S) sum [y log sigma(z) + (1-y) log(1 - sigma(z))]."""
    acts, _ = _forward(net, X)
    z = acts[-1]
    y = ((np.asarray(labels)[:, None] >> np.arange(4)) & 1).astype(np.float64)
    # -[y log s + (1-y) log(1-s)] = log(1 + e^z) - y z
    return float((np.logaddexp(0.0, z) - y * z).mean())


def grad(net, X, labels):
    """Gradient of loss() w.r.t. every parameter, packed in weights-file
    order (per layer W[out][in] then b[out])."""
    acts, pre = _forward(net, X)
    n = acts[0].shape[0]
    z = acts[-1]
    y = ((np.asarray(labels)[:, None] >> np.arange(4)) & 1).astype(np.float64)
    delta = (1.0 / (1.0 + np.exp(-z)) - y) / (n * 4)
    out = [None] * len(net.layers)
    for l in range(len(net.layers) - 1, -1, -1):
        W, _ = net.layers[l]
        out[l] = (delta.T @ acts[l], delta.sum(axis=0))
        if l > 0:
            delta = (delta @ W) * (pre[l - 1] > 0)
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in out])
