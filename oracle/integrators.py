"""Plain FP64 CPU oracle of second-order projective (outer) integrators for the
patch scheme.

TEST INFRASTRUCTURE ONLY: used by the tests; the product library never
imports it.  The paper integrates the macro level with forward Euler (eq.
(Extrapolation)) and names second-order Runge-Kutta and Adams-Bashforth outer
integrators as the higher-order alternatives (Section 1).  With
F(U, T) = (U^1 - U^0)/tau, the restricted change of the patch scheme from the
lift of U at time T (eq. (Time_Derivative)), the readings are:

* Heun (RK2):  U* = U_n + dt F(U_n, T_n) with the boundary data at T_{n+1};
               U_{n+1} = U_n + dt/2 (F(U_n, T_n) + F(U*, T_{n+1})),
               boundary data at T_{n+1};
* AB2:         U_{n+1} = U_n + dt (3/2 F(U_n, T_n) - 1/2 F(U_{n-1}, T_{n-1})),
               the first step of a run is a Heun step.

Each interior update is the oracle's projective step (orc_project) applied to
the combined change, so the boundary handling is the forward-Euler one.
Pinned in tests/test_oracle_integrators.py by the identity Heun step =
(U_n + FE(FE(U_n)))/2 on the interior, with FE the C oracle's own macro step,
and by observed temporal orders.
"""
from __future__ import annotations

import numpy as np

from . import Oracle


def patch_F(o: Oracle, U, t):
    """F of every patch: restricted change over tau (FP64 patch solver)."""
    sel = np.arange(o.n_patch, dtype=np.int32)
    return o.patch_dU(U, t, sel) / o.tau()


def step_euler(o: Oracle, U, t0, dt, n):
    """n forward-Euler projective steps (the paper's scheme) through F."""
    U = np.array(U, dtype=np.float64)
    tau = o.tau()
    for k in range(n):
        t = t0 + k * dt
        U = o.project(U, patch_F(o, U, t) * tau, t, dt, tau)
    return U


def step_heun(o: Oracle, U, t0, dt, n):
    """n Heun (RK2) projective steps."""
    U = np.array(U, dtype=np.float64)
    tau = o.tau()
    for k in range(n):
        t = t0 + k * dt
        F1 = patch_F(o, U, t)
        Us = o.project(U, F1 * tau, t, dt, tau)
        F2 = patch_F(o, Us, t + dt)
        U = o.project(U, 0.5 * (F1 + F2) * tau, t, dt, tau)
    return U


def step_ab2(o: Oracle, U, t0, dt, n):
    """n Adams-Bashforth-2 projective steps, the first one a Heun step."""
    U = np.array(U, dtype=np.float64)
    if n <= 0:
        return U
    tau = o.tau()
    F_prev = patch_F(o, U, t0)
    U = step_heun(o, U, t0, dt, 1)
    for k in range(1, n):
        t = t0 + k * dt
        F = patch_F(o, U, t)
        U = o.project(U, (1.5 * F - 0.5 * F_prev) * tau, t, dt, tau)
        F_prev = F
    return U
