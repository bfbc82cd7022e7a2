"""Pins of the oracle's Euler time integration (Sec. 4.4: third-order SSP
Runge-Kutta of Gottlieb and Shu, dt from the CFL condition).

The GPU steps are compared bit for bit with `oracle_step`, so its stage
combination has to be pinned by something other than itself:

* the temporal order: on a smooth periodic density wave with every stencil
  kept (all-smooth mask) and dx fixed, runs at CFL numbers halved in turn
  differ by C dt^3 from one another (the spatial error is the same in every
  run and cancels in the difference), so successive differences shrink by 8.
  A wrong stage weight of the kind that still sums to one (for example
  3/4 <-> 1/4 in the second stage, or 1/2, 1/2 in the last) leaves the
  scheme consistent but drops its order to 1 or 2;
* one step rebuilt from three right-hand sides with the Shu-Osher
  coefficients of the method written out here as fractions
  (u1 = u + dt L(u); u2 = 3/4 u + 1/4 u1 + 1/4 dt L(u1);
  u3 = 1/3 u + 2/3 u2 + 2/3 dt L(u2)), which must agree with oracle_step to
  rounding;
* the same step in Butcher form (nodes 0, 1, 1/2; weights 1/6, 1/6, 2/3),
  a different but equivalent statement of the method.

CPU only.
"""
from fractions import Fraction

import numpy as np

from conftest import balanced_net

import synth


def _density_wave(N, u=0.5, amp=0.2):
    x = (np.arange(N) + 0.5) / N
    rho = 1.0 + amp * np.sin(2 * np.pi * x)
    return synth.prim_to_cons(rho, u, 0.0, np.ones(N), ndim=1).reshape(3, 1, N)


def _run(o, U, cfl, t_end):
    t, n = 0.0, 0
    while t < t_end:
        U, t, _ = o.step(U, cfl, t, t_end)
        n += 1
    return U, n


def test_ssp_rk3_temporal_order(oracle_mod):
    N, t_end = 24, 0.4
    o = oracle_mod.Oracle(ndim=1, nx=N, bc=("periodic", "periodic"), mask_mode="smooth")
    U0 = _density_wave(N)
    cfls = (0.8, 0.4, 0.2, 0.1, 0.05)
    runs = [_run(o, U0.copy(), c, t_end) for c in cfls]
    assert runs[-1][1] >= 300  # many steps: the clipped last step is a small part
    diffs = np.array([np.abs(runs[k][0] - runs[k + 1][0]).sum() for k in range(len(cfls) - 1)])
    orders = np.log2(diffs[:-1] / diffs[1:])
    assert np.all(np.abs(orders - 3.0) < 0.1), (orders, diffs)


def _shu_osher_step(o, U, dt):
    q = {k: float(Fraction(*v)) for k, v in
         {"3/4": (3, 4), "1/4": (1, 4), "1/3": (1, 3), "2/3": (2, 3)}.items()}
    U1 = U + dt * o.rhs(U)
    U2 = q["3/4"] * U + q["1/4"] * U1 + q["1/4"] * dt * o.rhs(U1)
    return q["1/3"] * U + q["2/3"] * U2 + q["2/3"] * dt * o.rhs(U2)


def _butcher_step(o, U, dt):
    k1 = o.rhs(U)
    k2 = o.rhs(U + dt * k1)
    k3 = o.rhs(U + dt * (0.25 * k1 + 0.25 * k2))
    return U + dt * (k1 / 6.0 + k2 / 6.0 + (2.0 / 3.0) * k3)


def test_step_equals_three_rhs_combined(oracle_mod):
    cases = [
        (oracle_mod.Oracle(ndim=2, nx=20, ny=16, net=balanced_net(31)), synth.quadrants_2d(20, 16, seed=3), 0.4),
        (oracle_mod.Oracle(ndim=1, nx=64, bc=("transmissive", "transmissive"), net=balanced_net(32)),
         synth.riemann_1d(64, seed=4), 0.5),
    ]
    for o, U, cfl in cases:
        dt = o.dt(U, cfl)
        got, t, dt_step = o.step(U, cfl, 0.0, 0.0)
        assert dt_step == dt and t == dt
        for ref in (_shu_osher_step(o, U, dt), _butcher_step(o, U, dt)):
            # the masks of the intermediate stages are the step's own (same
            # stage states to rounding), so the results agree to rounding
            err = np.abs(got - ref)
            assert err.max() <= 1e-13 * np.abs(ref).max(), err.max()
        # a real change of state, far above that tolerance
        assert np.abs(got - U).max() > 1e-6 * np.abs(U).max()
