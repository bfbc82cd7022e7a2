"""The mixed-precision RHS at the benchmark's full size and launch
configuration (4096 x 4096 periodic four-quadrant state, the trained
classifier, the default guard bands): sampled cells and face masks against
the FP64 oracle, one by one."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def lib():
    import paper_2207_08500_gb300 as p
    from paper_2207_08500_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return p


@pytest.fixture(scope="module")
def state():
    return synth.quadrants_2d(N, N)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_full_size_mixed_sampled_against_oracle(lib, oracle_mod, state, prec):
    n = N
    net = oracle_mod.Net.load(lib.DEFAULT_WEIGHTS)
    g = lib.Neno6(ndim=2, nx=n, ny=n, precision=prec)
    o = oracle_mod.Oracle(ndim=2, nx=n, ny=n, net=net)
    d, m = g.rhs(torch.from_numpy(state).cuda(), want_mask=True)
    torch.cuda.synchronize()
    assert g.status() == 0
    d, m = d.cpu().numpy(), m.cpu().numpy()
    rng = np.random.default_rng(2)
    cells = rng.integers(0, n * n, 300)
    # the quadrant junctions, the periodic edges and the corners
    cells = np.concatenate([cells, [0, n - 1, n * (n - 1), n * n - 1, (n // 2) * n + n // 2,
                                    (n // 2 - 1) * n + n // 2 - 1, (n // 2) * n, n // 2]])
    ref = o.rhs_cells(state, cells)
    got = d.reshape(4, -1)[:, cells].T
    scale = np.abs(ref).max(axis=0)
    err = np.abs(got - ref).max(axis=0) / scale
    print("%s 4096^2: sampled max error per field / field scale: %s" % (prec, err))
    assert (err <= 2e-6).all(), err
    k = 300
    dirs = rng.integers(0, 2, k)
    faces = rng.integers(0, n + 1, k)
    lines = rng.integers(0, n, k)
    ref_m = o.face_masks(state, dirs, faces, lines)
    xblock = 4 * n * (n + 1)
    got_m = np.empty_like(ref_m)
    for r in range(k):
        for f in range(4):
            if dirs[r] == 0:
                idx = (f * n + lines[r]) * (n + 1) + faces[r]
            else:
                idx = xblock + (f * (n + 1) + faces[r]) * n + lines[r]
            got_m[r, f] = m[idx]
    assert np.array_equal(got_m, ref_m)
