"""Pins of the ADI micro solver of the oracle (Peaceman-Rachford splitting,
the scheme Section 4.1 runs inside the patches):

* a discrete cosine mode of the constant-coefficient patch operator with
  mirror (zero-flux) ghosts is an eigenvector of both line operators, so K ADI
  steps multiply it by the closed-form factor
  [(1 + h lx)(1 + h ly) / ((1 - h lx)(1 - h ly))]^K, h = dt / 2;
* with general coefficients (upwind convection, reaction, time-dependent
  source) the ADI burst converges to the exact solution of the semi-discrete
  patch problem w' = L w + r + (s(t) - s(T)) G, computed with a matrix
  exponential, at second order in dt when beta = 0 and first order when the
  mixed term is present (it is explicit);
* the summation-by-parts closed form of the restricted change holds for ADI
  bursts exactly as for forward Euler, for any step, also far beyond the
  explicit limit;
* the split (departure) form equals the literal burst.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import Oracle
from paper_2405_08764_gb300 import workloads as W


def _const_problem(**kw):
    p = W.base(n_xi=6, n_eta=5, m_xi=7, m_eta=9, h_ratio_xi=0.3, h_ratio_eta=0.2,
               M=(1.3, 0.0, 0.4), d_aff=(1.0, 0.0, 0.0), micro="adi")
    p.update(kw)
    return p


def _geom(p):
    dxi = p["h_ratio_xi"] * (p["box"][1] - p["box"][0]) / p["n_xi"] / (p["m_xi"] - 1)
    deta = p["h_ratio_eta"] * (p["box"][3] - p["box"][2]) / p["n_eta"] / (p["m_eta"] - 1)
    return dxi, deta


@pytest.mark.parametrize("j,l", [(1, 0), (0, 3), (2, 5), (6, 8), (3, 1)])
@pytest.mark.parametrize("K,dt_scale", [(1, 0.3), (3, 40.0)])
def test_cosine_mode_amplification(j, l, K, dt_scale):
    p = _const_problem()
    o = Oracle(p)
    nx, ny = p["m_xi"] - 1, p["m_eta"] - 1
    dxi, deta = _geom(p)
    al, ga = 1.3, 0.4
    dt = dt_scale / (2 * al / dxi ** 2 + 2 * ga / deta ** 2)
    a = np.arange(nx + 1)
    b = np.arange(ny + 1)
    w0 = np.outer(np.cos(l * math.pi * b / ny), np.cos(j * math.pi * a / nx))
    lx = -4 * al / dxi ** 2 * math.sin(j * math.pi / (2 * nx)) ** 2
    ly = -4 * ga / deta ** 2 * math.sin(l * math.pi / (2 * ny)) ** 2
    h = dt / 2
    rho = (1 + h * lx) * (1 + h * ly) / ((1 - h * lx) * (1 - h * ly))
    got = o.micro_patch(3, w0, None, 0.0, K, dt)
    np.testing.assert_allclose(got, rho ** K * w0, rtol=0, atol=1e-12)


def _general_problem(mixed: bool, conv: str = "upwind"):
    """Heterogeneous tensor diffusion on a tanh-stretched grid with affine
    velocity (upwind or central differences), reaction and an
    exponential-in-time source."""
    return W.base(n_xi=6, n_eta=6, m_xi=7, m_eta=7, map="tanh", map_p=(1.5, 2.0, 0.0, 0.0), conv=conv,
                  M=(1.0, 0.3 if mixed else 0.0, 0.6), d_aff=(0.02, 0.01, 0.005),
                  d_sin=(0.3, 1.0) if mixed else (0.0, 1.0),
                  va=(0.5, 0.4, 0.0), vb=(-0.3, 0.0, 0.2), f0=0.7,
                  src="exp_linear", src_p=(1.0, 0.5, -0.5), time="exp", tc=3.0,
                  micro="adi")


def _operator(o, p, dt):
    """L of the patch problem with zero edge data, from single forward-Euler
    steps of the oracle on unit vectors (L e_k = (FE(e_k) - e_k) / dt)."""
    pf = dict(p, micro="fe")
    of = Oracle(pf)
    n = o.mx * o.my
    L = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        L[:, k] = (of.micro_patch(0, e, None, 0.0, 1, dt).reshape(-1) - e) / dt
    return L


def _exact_burst(o, p, L, r, T, tau, tc):
    """w(tau) of w' = L w + r + (s(t) - s(T)) G, w(0) = 0, s(t) = exp(tc t),
    through the matrix exponential of the augmented system (w, s, 1)."""
    n = L.shape[0]
    xi, eta = o.micro_coords()
    G = np.array([o.coeffs(x, y)[6] for x, y in zip(xi[:n], eta[:n])])
    sT = math.exp(tc * T)
    A = np.zeros((n + 2, n + 2))
    A[:n, :n] = L
    A[:n, n] = G
    A[:n, n + 1] = r - sT * G
    A[n, n] = tc
    z0 = np.zeros(n + 2)
    z0[n] = sT
    z0[n + 1] = 1.0
    return (scipy.linalg.expm(tau * A) @ z0)[:n]


@pytest.mark.parametrize("mixed,order,conv", [(False, 2.0, "upwind"), (True, 1.0, "upwind"), (False, 2.0, "central")])
def test_adi_converges_to_the_semidiscrete_solution(mixed, order, conv):
    p = _general_problem(mixed, conv)
    o = Oracle(p)
    n = o.mx * o.my
    dt_fe = Oracle(dict(p, micro="fe")).dt_micro()
    L = _operator(o, p, dt_fe)
    rng = np.random.default_rng(11)
    r = rng.normal(size=n)
    T = 0.1
    tau = 40 * dt_fe
    ref = _exact_burst(o, p, L, r, T, tau, 3.0)
    errs = []
    for K in (5, 10, 20, 40):
        w = o.micro_patch(0, np.zeros(n), r, T, K, tau / K).reshape(-1)
        errs.append(np.linalg.norm(w - ref) / np.linalg.norm(ref))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert errs[-1] < 1e-2, errs
    assert all(abs(q - order) < 0.25 for q in rates[1:]), (rates, errs)


@pytest.mark.parametrize("K,scale", [(1, 0.5), (2, 30.0), (7, 200.0)])
@pytest.mark.parametrize("periodic", [0, 1])
def test_summation_by_parts_closed_form_with_adi(K, scale, periodic):
    """Constant alpha, gamma, no convection, reaction or source, LIFTED
    restriction: dU = tau (alpha/Dxi^2 sum_q w_q (U_{i+1,q} - 2 U_{i,q} + U_{i-1,q})
    + gamma/Deta^2 sum_p w_p (...)) with w_{+-1} = (h^2/12 + d^2/6) / (2 Delta^2),
    w_0 = 1 - 2 w_{+-1}, whatever the micro dynamics."""
    p = W.base(n_xi=7, n_eta=6, periodic_xi=periodic, m_xi=7, m_eta=5, h_ratio_xi=0.35,
               h_ratio_eta=0.25, M=(0.8, 0.0, 1.7), d_aff=(1.0, 0.0, 0.0), micro="adi",
               box=(0.0, 2.0 * math.pi, 0.0, 1.0) if periodic else (0.0, 1.0, 0.0, 1.0))
    o = Oracle(p)
    dt = scale * Oracle(dict(p, micro="fe")).dt_micro()
    U = np.random.default_rng(5).normal(size=o.n_macro)
    burst = o.burst(U, 0.0, K, dt)
    dU = o.restrict(U, burst)
    tau = K * dt
    Ug = U.reshape(o.nyp, o.nxp)
    I, J = o.patch_nodes()
    Dx = (p["box"][1] - p["box"][0]) / p["n_xi"]
    Dy = (p["box"][3] - p["box"][2]) / p["n_eta"]
    hx, hy = p["h_ratio_xi"] * Dx, p["h_ratio_eta"] * Dy
    dx, dy = hx / (p["m_xi"] - 1), hy / (p["m_eta"] - 1)
    wx1 = (hx ** 2 / 12 + dx ** 2 / 6) / (2 * Dx ** 2)
    wy1 = (hy ** 2 / 12 + dy ** 2 / 6) / (2 * Dy ** 2)
    wx = {-1: wx1, 0: 1 - 2 * wx1, 1: wx1}
    wy = {-1: wy1, 0: 1 - 2 * wy1, 1: wy1}
    want = np.zeros(o.n_patch)
    for k, (i, j) in enumerate(zip(I, J)):
        def u(ii, jj):
            return Ug[jj, ii % o.nxp] if periodic else Ug[jj, ii]
        sx = sum(wy[q] * (u(i + 1, j + q) - 2 * u(i, j + q) + u(i - 1, j + q)) for q in (-1, 0, 1))
        sy = sum(wx[q] * (u(i + q, j + 1) - 2 * u(i + q, j) + u(i + q, j - 1)) for q in (-1, 0, 1))
        want[k] = tau * (0.8 * sx / Dx ** 2 + 1.7 * sy / Dy ** 2)
    np.testing.assert_allclose(dU, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("prob", ["paper", "tensor", "annulus"])
def test_adi_split_burst_equals_literal_burst(prob):
    if prob == "paper":
        p = W.paper_cdr(True, lam=0.3, n=6, m=9)
    elif prob == "tensor":
        p = _general_problem(True)
    else:
        p = W.paper_annulus(n_theta=8, n_r=5, m=7)
    p = dict(p, micro="adi")
    o = Oracle(p)
    dt = 25 * o.dt_micro()
    U = o.init_field() + 0.1 * np.random.default_rng(2).normal(size=o.n_macro)
    u0, _ = o.lift(U)
    w = o.burst(U, 0.05, 3, dt, form="split")
    u = o.burst(U, 0.05, 3, dt, form="literal")
    np.testing.assert_allclose(u0 + w, u, rtol=0, atol=1e-12 * np.abs(u).max())
    np.testing.assert_allclose(o.restrict(U, w, "split"), o.restrict(U, u, "literal"),
                               rtol=0, atol=1e-12 * np.abs(u).max())


def test_fixed_micro_step_overrides_the_cfl_rule():
    p = W.paper_cdr(False, lam=0.1, n=6, m=11)
    o = Oracle(dict(p, micro="adi", dt_micro=5e-7))
    assert o.dt_micro() == 5e-7
    assert Oracle(p).dt_micro() < 1e-6
