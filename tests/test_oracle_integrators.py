"""Pins of the second-order projective integrators (oracle/integrators.py):
the Heun step against two forward-Euler steps of the C oracle's own macro step
(an identity of the method), AB2's first step, and the observed temporal
orders on the manufactured solution (first order for forward Euler, second
for Heun and AB2), measured against a fine-step Heun reference on the same
patch grid so that the spatial error cancels."""
import math

import numpy as np

from oracle import Oracle
from oracle import integrators as R
from paper_2405_08764_gb300 import workloads as W


def _interior(o, U):
    I, J = o.patch_nodes()
    return np.asarray(U).reshape(o.nyp, o.nxp)[J, I]


def test_heun_step_is_the_mean_of_the_field_and_two_euler_steps():
    p = W.c2_heterogeneous(n=10, m=7, n_macro=2)
    o = Oracle(p)
    U0 = o.init_field() + 0.01 * np.random.default_rng(3).normal(size=o.n_macro)
    U0 = o.apply_bc(U0, 0.0)
    dt = 0.5 * o.dt_macro()
    got = R.step_heun(o, U0, 0.0, dt, 1)
    fe1 = o.step(U0, 0.0, dt, 1)              # the C oracle's own macro step
    fe2 = o.step(fe1, dt, dt, 1)
    want = 0.5 * (_interior(o, U0) + _interior(o, fe2))
    np.testing.assert_allclose(_interior(o, got), want, rtol=0, atol=1e-13 * np.abs(want).max())
    # boundary data at T_{n+1}, as after one Euler step
    bnd = ~np.isin(np.arange(o.n_macro), _nodes(o))
    np.testing.assert_array_equal(got[bnd], fe1[bnd])
    # the Euler path through F equals the C oracle's step
    np.testing.assert_allclose(R.step_euler(o, U0, 0.0, dt, 2), o.step(U0, 0.0, dt, 2), rtol=0,
                               atol=1e-13 * np.abs(U0).max())


def _nodes(o):
    I, J = o.patch_nodes()
    return J * o.nxp + I


def test_ab2_starts_with_a_heun_step():
    p = W.c1_manufactured(n=8, m=5)
    o = Oracle(p)
    U0 = o.init_field()
    dt = 0.01
    np.testing.assert_array_equal(R.step_ab2(o, U0, 0.0, dt, 1), R.step_heun(o, U0, 0.0, dt, 1))
    # second step: U2 = U1 + dt (3/2 F1 - 1/2 F0) on the interior
    U1 = R.step_heun(o, U0, 0.0, dt, 1)
    F0 = R.patch_F(o, U0, 0.0)
    F1 = R.patch_F(o, U1, dt)
    U2 = R.step_ab2(o, U0, 0.0, dt, 2)
    np.testing.assert_allclose(_interior(o, U2), _interior(o, U1) + dt * (1.5 * F1 - 0.5 * F0),
                               rtol=0, atol=1e-13 * np.abs(U1).max())


def _order(step, o, U0, T, ref):
    errs = []
    for n in (4, 8, 16):
        U = step(o, U0, 0.0, T / n, n)
        errs.append(np.linalg.norm(_interior(o, U) - ref))
    return [math.log2(errs[k] / errs[k + 1]) for k in range(2)], errs


def test_temporal_orders_on_the_manufactured_solution():
    """Large macro steps (up to the explicit bound) so that the time error
    dominates; the reference is Heun with 128 steps on the same grid."""
    p = W.c1_manufactured(n=8, m=5)
    o = Oracle(p)
    U0 = o.init_field()
    T = 16 * 0.9 * o.dt_macro()
    ref = _interior(o, R.step_heun(o, U0, 0.0, T / 128, 128))
    fe, _ = _order(R.step_euler, o, U0, T, ref)
    heun, _ = _order(R.step_heun, o, U0, T, ref)
    ab2, _ = _order(R.step_ab2, o, U0, T, ref)
    assert all(0.8 <= q <= 1.3 for q in fe), fe
    assert all(q >= 1.8 for q in heun), heun
    assert all(q >= 1.7 for q in ab2), ab2
