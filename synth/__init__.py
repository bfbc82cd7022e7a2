"""Seeded synthetic inputs for the NENO6 Euler workloads.

This module holds no arithmetic of the method: it only draws initial states,
cotangents, perturbation directions and classifier stencils.  Both the CUDA
path (tests, bench) and the oracle consume its output; neither side imports
the other.  Everything is generated on the host with numpy's PCG64 from an
explicit seed, so both sides see identical bits.

State arrays are float64 [nv][ny][nx] with conserved variables
(rho, rho*u, [rho*v], E), E = p/(gamma-1) + rho*|u|^2/2, cell centres at
x_i = (i + 1/2) dx.
"""
import math

import numpy as np

BASE_SEED = 20220717


def prim_to_cons(rho, u, v, p, gamma=1.4, ndim=2):
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + (v * v if ndim == 2 else 0.0))
    if ndim == 1:
        return np.stack([rho, rho * u, E])
    return np.stack([rho, rho * u, rho * v, E])


def _sound(rho, p, gamma):
    return math.sqrt(gamma * p / rho)


def _no_vacuum(a, b, gamma, margin=0.5):
    """Pressure-positivity condition of the exact Riemann problem between
    primitive states a=(rho,un,p) (left) and b (right), with a margin."""
    ca, cb = _sound(a[0], a[2], gamma), _sound(b[0], b[2], gamma)
    return (b[1] - a[1]) < margin * 2.0 / (gamma - 1.0) * (ca + cb)


def riemann_1d(n=400, seed=BASE_SEED + 0, gamma=1.4):
    """1D Riemann data on [0,1], jump at x = 0.5: rho ~ U[0.1,1],
    u ~ U[-0.5,0.5], p ~ U[0.1,1] on each side (redrawn if the pair would
    open a vacuum).  Returns U [3][1][n]."""
    rng = np.random.default_rng(seed)
    while True:
        L = (rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0))
        R = (rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0))
        if _no_vacuum(L, R, gamma):
            break
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    rho = np.where(left, L[0], R[0])
    u = np.where(left, L[1], R[1])
    p = np.where(left, L[2], R[2])
    return prim_to_cons(rho, u, 0.0, p, gamma, ndim=1).reshape(3, 1, n)


def quadrants_2d(nx, ny, seed=BASE_SEED + 1, gamma=1.4, amp=0.01, modes=8):
    """Four piecewise-constant quadrants on the periodic unit square:
    rho, p ~ U[0.1,1.5], u, v ~ U[-0.8,0.8] per quadrant (redrawn until no
    pair of neighbouring quadrants, across the periodic wrap too, would open a
    vacuum), times a density perturbation
        1 + amp * sum_{k=1..modes} a_k sin(2 pi k s_k + phi_k) / modes
    with a_k ~ U[0,1], phi_k ~ U[0, 2 pi) and s_k = x or y (seeded per mode).
    Returns U [4][ny][nx]."""
    rng = np.random.default_rng(seed)
    while True:
        Q = [(rng.uniform(0.1, 1.5), rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8),
              rng.uniform(0.1, 1.5)) for _ in range(4)]
        # quadrant index q = 2*(y>=0.5) + (x>=0.5); x neighbours (0,1),(2,3), y (0,2),(1,3)
        ok = True
        for a, b in ((0, 1), (2, 3)):
            for l, r in ((a, b), (b, a)):
                ok &= _no_vacuum((Q[l][0], Q[l][1], Q[l][3]), (Q[r][0], Q[r][1], Q[r][3]), gamma)
        for a, b in ((0, 2), (1, 3)):
            for l, r in ((a, b), (b, a)):
                ok &= _no_vacuum((Q[l][0], Q[l][2], Q[l][3]), (Q[r][0], Q[r][2], Q[r][3]), gamma)
        if ok:
            break
    a_k = rng.uniform(0.0, 1.0, modes)
    phi = rng.uniform(0.0, 2 * math.pi, modes)
    along_y = rng.integers(0, 2, modes)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    q = 2 * (Y >= 0.5) + (X >= 0.5)
    prim = np.array(Q)[q]  # [ny, nx, 4]
    pert = np.zeros_like(X)
    for k in range(modes):
        s = Y if along_y[k] else X
        pert += a_k[k] * np.sin(2 * math.pi * (k + 1) * s + phi[k])
    rho = prim[..., 0] * (1.0 + amp * pert / modes)
    return prim_to_cons(rho, prim[..., 1], prim[..., 2], prim[..., 3], gamma)


def smooth_2d(nx, ny, seed=BASE_SEED + 11, gamma=1.4, amp=0.05):
    """Smooth periodic state with every field perturbed (no ties between
    neighbouring cells; used by the differentiation tests)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    def field(base):
        # separable modes with random phases: no lattice symmetry, hence no
        # exact ties between cells
        f = np.full_like(X, base)
        for _ in range(3):
            kx, ky = rng.integers(1, 4, 2)
            f += amp * rng.uniform(0.2, 1.0) * (
                np.sin(2 * math.pi * kx * X + rng.uniform(0, 2 * math.pi))
                * np.cos(2 * math.pi * ky * Y + rng.uniform(0, 2 * math.pi)))
        return f
    rho, u, v, p = field(1.0), field(0.3), field(-0.2), field(1.0)
    return prim_to_cons(rho, u, v, p, gamma)


def noisy(U, seed, rel=1e-3, gamma=1.4):
    """Multiply density, velocity and pressure by (1 + rel*N(0,1)) per cell
    (breaks exact ties in piecewise-constant data)."""
    rng = np.random.default_rng(seed)
    nv = U.shape[0]
    rho = U[0]
    u = U[1] / rho
    v = U[2] / rho if nv == 4 else 0.0
    E = U[-1]
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + (v * v if nv == 4 else 0.0)))
    g = lambda a: a * (1.0 + rel * rng.standard_normal(rho.shape))
    rho, u, p = g(rho), g(u), g(p)
    if nv == 4:
        v = g(v)
    return prim_to_cons(rho, u, v, p, gamma, ndim=2 if nv == 4 else 1).reshape(U.shape)


def oblique_shock_2d(nx, ny, seed=BASE_SEED + 4, gamma=1.4, blobs=16):
    """Oblique shock in [0, nx/ny] x [0, 1]: upstream rho=1.4, p=1 (c=1) moving
    in +x at Mach M ~ U[2,10]; shock line through (x0, 0) at angle
    beta ~ U[30, 60] degrees; downstream state from the normal-shock
    (Rankine-Hugoniot) relations at M_n = M sin(beta), tangential velocity
    unchanged; plus Gaussian density blobs of relative amplitude <= 0.2."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(2.0, 10.0)
    beta = math.radians(rng.uniform(30.0, 60.0))
    Lx = nx / ny
    x0 = rng.uniform(0.1, 0.3) * Lx
    rho1, p1 = gamma, 1.0
    c1 = 1.0
    Mn = M * math.sin(beta)
    r = (gamma + 1) * Mn * Mn / ((gamma - 1) * Mn * Mn + 2)
    rho2 = rho1 * r
    p2 = p1 * (1 + 2 * gamma / (gamma + 1) * (Mn * Mn - 1))
    n_ = (math.sin(beta), -math.cos(beta))
    t_ = (math.cos(beta), math.sin(beta))
    w1 = M * c1 * math.sin(beta)
    wt = M * c1 * math.cos(beta)
    w2 = w1 / r
    u2 = w2 * n_[0] + wt * t_[0]
    v2 = w2 * n_[1] + wt * t_[1]
    x = (np.arange(nx) + 0.5) / ny
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    down = (X - x0) * n_[0] + Y * n_[1] > 0
    rho = np.where(down, rho2, rho1)
    u = np.where(down, u2, M * c1)
    v = np.where(down, v2, 0.0)
    p = np.where(down, p2, p1)
    for _ in range(blobs):
        cx, cy = rng.uniform(0, Lx), rng.uniform(0, 1)
        w = rng.uniform(0.01, 0.05)
        a = rng.uniform(-0.2, 0.2)
        rho = rho * (1 + a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * w * w)))
    return prim_to_cons(rho, u, v, p, gamma)


def mlp_stencils(n, seed=BASE_SEED + 3):
    """n six-point stencils: the first half a*sin(k*x + phi) sampled at six
    consecutive points (a ~ U[0.1,2], k*dx ~ U[0.05,1.5], phi ~ U[0,2pi)),
    the second half a step of height h ~ U[-2,2] on a base b ~ U[-1,1] at a
    seeded face position 1..5.  Returns float64 [n][6]."""
    rng = np.random.default_rng(seed)
    h = n // 2
    j = np.arange(6)
    a = rng.uniform(0.1, 2.0, h)[:, None]
    kdx = rng.uniform(0.05, 1.5, h)[:, None]
    phi = rng.uniform(0, 2 * math.pi, h)[:, None]
    smooth = a * np.sin(kdx * j[None, :] + phi)
    m = n - h
    b = rng.uniform(-1.0, 1.0, m)[:, None]
    hh = rng.uniform(-2.0, 2.0, m)[:, None]
    pos = rng.integers(1, 6, m)[:, None]
    step = b + hh * (j[None, :] >= pos)
    return np.ascontiguousarray(np.concatenate([smooth, step]), dtype=np.float64)


def normal(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def random_states(n, seed, ndim=2, gamma=1.4):
    """n random physical cell states, columns [nv][n]."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 2.0, n)
    u = rng.uniform(-1.0, 1.0, n)
    v = rng.uniform(-1.0, 1.0, n)
    p = rng.uniform(0.1, 2.0, n)
    return prim_to_cons(rho, u, v, p, gamma, ndim=ndim)
