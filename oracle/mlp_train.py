"""Mini-batch Adam training of the classifier, FP64 (oracle side).

Test infrastructure.  Sec. 3.3 and Table 2: Adam (Kingma & Ba, Algorithm 1,
with its default hyper-parameters beta1 = 0.9, beta2 = 0.999, epsilon = 1e-8)
on the mean binary cross entropy of Eq. (Crossentropy), one update per
mini-batch, the batches taken in the order of a given permutation.  Written
from the definition:

    m_t = beta1 m_{t-1} + (1 - beta1) g_t
    v_t = beta2 v_{t-1} + (1 - beta2) g_t^2
    theta_t = theta_{t-1} - lr (m_t / (1 - beta1^t)) / (sqrt(v_t / (1 - beta2^t)) + epsilon)

with g_t the gradient of mlp_grad.loss on the t-th batch (mlp_grad.grad).
Pinned in tests/test_oracle_mlp_train.py by hand-computed iterates on a
one-parameter quadratic and by the first-step closed form.
"""
import numpy as np

from . import mlp_grad
from .weights import Net

BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def adam_step(theta, g, m, v, t, lr, beta1=BETA1, beta2=BETA2, eps=EPS):
    """One Adam update (step number t >= 1) of the arrays theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def unpack(net, p):
    """A Net with the layer shapes of `net` and the packed parameters p."""
    layers, o = [], 0
    for W, b in net.layers:
        layers.append((p[o:o + W.size].reshape(W.shape).copy(), p[o + W.size:o + W.size + b.size].copy()))
        o += W.size + b.size
    return Net(layers)


def train(net, X, labels, perm, batch, lr, m=None, v=None, t0=0):
    """Adam steps over perm in batches; returns (packed parameters, m, v,
    list of each batch's loss before its update)."""
    p = net.packed().astype(np.float64)
    m = np.zeros_like(p) if m is None else np.asarray(m, dtype=np.float64).copy()
    v = np.zeros_like(p) if v is None else np.asarray(v, dtype=np.float64).copy()
    X = np.asarray(X, dtype=np.float64)
    labels = np.asarray(labels)
    perm = np.asarray(perm)
    losses = []
    for k, s0 in enumerate(range(0, len(perm), batch)):
        idx = perm[s0:s0 + batch]
        cur = unpack(net, p)
        losses.append(mlp_grad.loss(cur, X[idx], labels[idx]))
        g = mlp_grad.grad(cur, X[idx], labels[idx])
        p, m, v = adam_step(p, g, m, v, t0 + k + 1, lr)
    return p, m, v, losses
