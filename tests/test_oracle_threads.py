"""The oracle's face loops run under OpenMP; every face's arithmetic and the
place its result goes do not depend on the thread count, so a threaded
right-hand side (masks, dU/dt), step and adjoint must equal the one-thread
results bit for bit.  CPU only."""
import numpy as np

from conftest import balanced_net

import synth


def test_threaded_oracle_is_bit_identical(oracle_mod):
    net = balanced_net(41)
    U = synth.smooth_2d(40, 36, seed=5)  # a random classifier stays stable on smooth data
    o = oracle_mod.Oracle(ndim=2, nx=40, ny=36, net=net)
    full = oracle_mod.set_threads(0)
    out = {}
    for th in sorted({1, max(2, full)}):
        oracle_mod.set_threads(th)
        d, m = o.rhs(U, want_mask=True)
        s, _, _ = o.step(U, 0.4)
        _, jv = o.jvp(U, synth.normal(U.shape, seed=6), m)
        assert np.isfinite(s).all() and 0 < np.unpackbits(m).mean() < 1
        out[th] = (d, m, s, jv)
    oracle_mod.set_threads(full)
    a, b = out.values()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
