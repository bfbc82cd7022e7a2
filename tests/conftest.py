import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def balanced_net(seed=1, widths=(6, 64, 32, 16, 8, 4)):
    """Random classifier whose output biases are shifted so that each logit is
    positive on about half of a seeded stencil sample: parity tests then
    exercise every mask pattern, including the all-discarded fallback."""
    import oracle
    import synth
    net = oracle.Net.random(widths, seed=seed)
    X = synth.mlp_stencils(4096, seed=seed + 100)
    o = oracle.Oracle(ndim=1, nx=8, net=net)
    _, logits = o.classify(X)
    W, b = net.layers[-1]
    net.layers[-1] = (W, b - np.median(logits, axis=0))
    return net


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
