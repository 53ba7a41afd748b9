"""Pins for the oracle's patch scheme (Section 3): edge data, lift, ghost-point
burst, restriction and projection, against closed forms and identities that
hold for the method exactly."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W

RNG = np.random.default_rng(99)


def _aniso(**kw):
    p = W.base(n_xi=5, n_eta=4, box=(0.0, 1.3, -0.2, 0.9), m_xi=7, m_eta=5,
               h_ratio_xi=0.3, h_ratio_eta=0.45, k_micro=9)
    p.update(kw)
    return p


def _geom(o, p):
    s = o.s
    Dx = (s.xi1 - s.xi0) / s.n_xi
    Dy = (s.eta1 - s.eta0) / s.n_eta
    hx, hy = s.h_ratio_xi * Dx, s.h_ratio_eta * Dy
    return Dx, Dy, hx, hy, hx / (s.m_xi - 1), hy / (s.m_eta - 1)


def _stencil(o, U, p):
    i, j = o.patch_nodes()
    i, j = i[p], j[p]
    Ug = U.reshape(o.nyp, o.nxp)
    return np.array([[Ug[j + q, (i + pp) % o.nxp] for q in (-1, 0, 1)] for pp in (-1, 0, 1)])


def test_edge_data_is_the_derivative_of_the_lagrange_interpolant(orc):
    """Eq. (edge) equals d/dxi (resp. d/deta) of the biquadratic interpolant of
    eq. (Lagrange_2D) at the patch edges; interpolant rebuilt here with numpy's
    polynomial fit through three nodes (exact interpolation)."""
    p = _aniso()
    o = orc.Oracle(p)
    U = RNG.normal(size=o.n_macro)
    _, edge = o.lift(U)
    Dx, Dy, hx, hy, dx, dy = _geom(o, p)
    nodes_x, nodes_y = np.array([-Dx, 0, Dx]), np.array([-Dy, 0, Dy])
    for pch in (0, 5, o.n_patch - 1):
        st = _stencil(o, U, pch)
        for b in range(-1, o.my + 1):
            t = -0.5 * hy + b * dy
            col = np.array([np.polyval(np.polyfit(nodes_y, st[pp], 2), t) for pp in range(3)])
            dpoly = np.poly1d(np.polyder(np.polyfit(nodes_x, col, 2)))
            np.testing.assert_allclose(edge[pch, 0, b + 1], dpoly(-hx / 2), rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose(edge[pch, 1, b + 1], dpoly(hx / 2), rtol=1e-9, atol=1e-9)
        for a in range(-1, o.mx + 1):
            s = -0.5 * hx + a * dx
            row = np.array([np.polyval(np.polyfit(nodes_x, st[:, q], 2), s) for q in range(3)])
            dpoly = np.poly1d(np.polyder(np.polyfit(nodes_y, row, 2)))
            np.testing.assert_allclose(edge[pch, 2, a + 1], dpoly(-hy / 2), rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose(edge[pch, 3, a + 1], dpoly(hy / 2), rtol=1e-9, atol=1e-9)


def test_lift_is_quadratic_with_patch_average_U(orc):
    """Eqs. (Lifting), (C_0): the lifted field is a quadratic whose continuous
    patch average is U_ij (the purpose of C_0), and whose trapezoid average is
    U_ij + (dxi^2 U_xixi + deta^2 U_etaeta) / 12."""
    p = _aniso()
    o = orc.Oracle(p)
    U = RNG.normal(size=o.n_macro)
    u0, _ = o.lift(U)
    Dx, Dy, hx, hy, dx, dy = _geom(o, p)
    s = -0.5 * hx + np.arange(o.mx) * dx
    t = -0.5 * hy + np.arange(o.my) * dy
    S, T = np.meshgrid(s, t)
    A = np.stack([np.ones_like(S), S, T, S * S, S * T, T * T], -1).reshape(-1, 6)
    wx = np.ones(o.mx); wx[[0, -1]] = 0.5
    wy = np.ones(o.my); wy[[0, -1]] = 0.5
    for pch in range(o.n_patch):
        coef, res, *_ = np.linalg.lstsq(A, u0[pch].ravel(), rcond=None)
        assert np.abs(A @ coef - u0[pch].ravel()).max() < 1e-12
        st = _stencil(o, U, pch)
        mean = coef[0] + coef[3] * hx * hx / 12 + coef[5] * hy * hy / 12
        np.testing.assert_allclose(mean, st[1, 1], rtol=1e-12, atol=1e-12)
        trap = (wy[:, None] * wx[None, :] * u0[pch]).sum() / ((o.mx - 1) * (o.my - 1))
        Uxx = (st[2, 1] - 2 * st[1, 1] + st[0, 1]) / Dx ** 2
        Uyy = (st[1, 2] - 2 * st[1, 1] + st[1, 0]) / Dy ** 2
        np.testing.assert_allclose(trap, st[1, 1] + (dx * dx * Uxx + dy * dy * Uyy) / 12,
                                   rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("K,cfl", [(1, 0.4), (9, 0.4), (37, 0.9)])
@pytest.mark.parametrize("periodic", [0, 1])
def test_summation_by_parts_closed_form(orc, K, cfl, periodic):
    """For constant alpha, gamma and no other terms, the trapezoid sum of the
    ghost-point Laplacian telescopes to the edge data, so in LIFTED mode
      F = (alpha/Dxi^2) sum_q w_q (U_{i+1,q} - 2U_{i,q} + U_{i-1,q})
        + (gamma/Deta^2) sum_p w_p (U_{p,j+1} - 2U_{p,j} + U_{p,j-1}),
    w_{+-1} = (h^2/12 + d^2/6)/(2 Delta^2), w_0 = 1 - 2 w_{+-1}, for ANY number of
    micro steps and any micro step.  Pins eq. (edge), the ghost points, the
    burst, the trapezoid restriction and the time-derivative estimate."""
    p = _aniso(M=(0.8, 0.0, 1.7), d_aff=(1.0, 0.0, 0.0), k_micro=K, cfl_micro=cfl,
               periodic_xi=periodic)
    o = orc.Oracle(p)
    U = RNG.normal(size=o.n_macro)
    dt = o.dt_micro()
    dU = o.restrict(U, o.burst(U, 0.0, K, dt))
    F = dU / (K * dt)
    Dx, Dy, hx, hy, dx, dy = _geom(o, p)
    wxn = (hx * hx / 12 + dx * dx / 6) / (2 * Dx * Dx)
    wyn = (hy * hy / 12 + dy * dy / 6) / (2 * Dy * Dy)
    wx = np.array([wxn, 1 - 2 * wxn, wxn])
    wy = np.array([wyn, 1 - 2 * wyn, wyn])
    for pch in range(o.n_patch):
        st = _stencil(o, U, pch)
        d2x = st[2] - 2 * st[1] + st[0]          # over q
        d2y = st[:, 2] - 2 * st[:, 1] + st[:, 0]  # over p
        want = 0.8 / Dx ** 2 * (wy @ d2x) + 1.7 / Dy ** 2 * (wx @ d2y)
        np.testing.assert_allclose(F[pch], want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def test_macro_restriction_adds_the_trapezoid_bias(orc):
    """Reading G4: the paper-literal reference U^0 = U_ij differs from the lifted
    reference by exactly (dxi^2 U_xixi + deta^2 U_etaeta)/12."""
    p = _aniso(M=(0.8, 0.1, 1.7), va=(0.3, 0, 0), vb=(-0.2, 0, 0))
    o1 = orc.Oracle(p)
    o2 = orc.Oracle(dict(p, restrict="macro"))
    U = RNG.normal(size=o1.n_macro)
    dt = o1.dt_micro()
    d1 = o1.restrict(U, o1.burst(U, 0.0, 5, dt))
    d2 = o2.restrict(U, o2.burst(U, 0.0, 5, dt))
    Dx, Dy, hx, hy, dx, dy = _geom(o1, p)
    for pch in range(o1.n_patch):
        st = _stencil(o1, U, pch)
        bias = (dx * dx * (st[2, 1] - 2 * st[1, 1] + st[0, 1]) / Dx ** 2
                + dy * dy * (st[1, 2] - 2 * st[1, 1] + st[1, 0]) / Dy ** 2) / 12
        np.testing.assert_allclose(d2[pch] - d1[pch], bias, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("prob", ["c1", "tensor", "annulus"])
def test_split_burst_equals_literal_burst(orc, prob):
    """Reading: the burst is evolved as u = u_lift + w.  Because u_lift and the
    edge data are fixed over the burst, this is an exact rewriting of the
    literal forward-Euler recursion on u; the two agree to rounding."""
    if prob == "c1":
        p = W.c1_manufactured()
    elif prob == "tensor":
        p = _aniso(map="tanh", map_p=(1.5, 2.0, 0, 0), M=(1.0, 0.3, 0.8), d_aff=(0.2, 0.1, 0.0),
                   va=(1.0, 0.5, 0.0), vb=(-0.5, 0.0, 0.5), f0=0.4, src="mms_sinprod",
                   time="exp", tc=-1.0)
    else:
        p = W.paper_annulus()
    o = orc.Oracle(p)
    U = o.init_field() if prob != "tensor" else 1.0 + 0.1 * RNG.normal(size=o.n_macro)
    dt = o.dt_micro()
    K = o.s.k_micro
    u0, _ = o.lift(U)
    w = o.burst(U, 0.3, K, dt, "split")
    u = o.burst(U, 0.3, K, dt, "literal")
    np.testing.assert_allclose(u0 + w, u, rtol=0, atol=1e-13 * np.abs(u).max())
    d_s = o.restrict(U, w, "split")
    d_l = o.restrict(U, u, "literal")
    np.testing.assert_allclose(d_s, d_l, rtol=0, atol=1e-12 * np.abs(u).max())


def test_step_composes_burst_restrict_project(orc):
    p = _aniso(map="tanh", map_p=(2.0, 1.0, 0, 0), M=(1.0, 0.2, 0.5), va=(0.5, 0.2, 0.0),
               vb=(0.3, 0.0, 0.0), src="mms_sinprod", time="exp", tc=-1.0, sol="sinprod_decay")
    o = orc.Oracle(p)
    U = o.apply_bc(RNG.normal(size=o.n_macro), 0.2)
    dt, dtm = o.dt_micro(), 0.3 * o.dt_macro()
    tau = o.s.k_micro * dt
    w = o.burst(U, 0.2, o.s.k_micro, dt)
    U1 = o.project(U, o.restrict(U, w), 0.2, dtm, tau)
    U2 = o.step(U, 0.2, dtm, 1, dt)
    np.testing.assert_array_equal(U1, U2)


@pytest.mark.parametrize("conv", ["upwind", "central"])
def test_step_sizes_closed_form(orc, conv):
    """Identity map with constant coefficients (cross term, convection,
    reaction): the micro step is cfl over the forward-Euler rate bound of the
    micro grid, 2 alpha/dxi^2 + 2 gamma/deta^2 + |beta|/(dxi deta) + |phi|
    (+ |nu|/dxi + |omega|/deta with upwind convection; central differences
    drop them), and the macro step half the inverse of the same bound on the
    macro grid with the convection terms always in."""
    d11, d12, d22, v1, v2, f0 = 0.05, 0.015, 0.08, 0.9, -1.3, -0.6
    cfl, hr, m = 0.4, 0.2, 7
    p = W.base(n_xi=8, n_eta=6, m_xi=m, m_eta=m, h_ratio_xi=hr, h_ratio_eta=hr, cfl_micro=cfl, conv=conv,
               M=(d11, d12, d22), d_aff=(1.0, 0.0, 0.0), va=(v1, 0.0, 0.0), vb=(v2, 0.0, 0.0), f0=f0)
    o = orc.Oracle(p)
    Dx, Dy = 1 / 8, 1 / 6
    dx, dy = hr * Dx / (m - 1), hr * Dy / (m - 1)
    beta = 2 * d12
    r_mic = 2 * d11 / dx ** 2 + 2 * d22 / dy ** 2 + abs(beta) / (dx * dy) + abs(f0)
    if conv == "upwind":
        r_mic += abs(v1) / dx + abs(v2) / dy
    r_mac = 2 * d11 / Dx ** 2 + 2 * d22 / Dy ** 2 + abs(beta) / (Dx * Dy) + abs(v1) / Dx + abs(v2) / Dy + abs(f0)
    assert o.dt_micro() == pytest.approx(cfl / r_mic, rel=1e-13)
    assert o.dt_macro() == pytest.approx(0.5 / r_mac, rel=1e-13)


def test_sampled_patches_equal_the_full_passes(orc):
    """patch_dU on a shuffled subset of patches returns, for each selected
    patch, the restricted change that the full lift -> burst -> restrict passes
    give that patch."""
    p = W.c2_heterogeneous(n=7, m=5, n_macro=1)
    o = orc.Oracle(p)
    U = o.init_field() + np.random.default_rng(4).normal(size=o.n_macro) * 0.1
    t, K, dt = 0.3, p["k_micro"], o.dt_micro()
    full = o.restrict(U, o.burst(U, t, K, dt))
    sel = np.random.default_rng(5).permutation(o.n_patch)[:17]
    np.testing.assert_allclose(o.patch_dU(U, t, sel), full[sel], rtol=1e-13, atol=1e-15 * np.abs(full).max())


@pytest.mark.parametrize("periodic", [0, 1])
def test_boundary_data_on_exactly_the_boundary_nodes(orc, periodic):
    """Dirichlet data at time t go to the first and last node rows and, unless
    xi is periodic, the first and last node columns: the exact solution at each
    node's physical point (zero without one); interior nodes are untouched."""
    if periodic:
        p = W.paper_annulus(n_theta=12, n_r=6, m=5)
    else:
        p = W.paper_cdr(False, lam=0.3, n=7, m=5)
    o = orc.Oracle(p)
    U = np.random.default_rng(6).normal(size=o.n_macro)
    t = 0.45
    V = o.apply_bc(U, t).reshape(o.nyp, o.nxp)
    bnd = np.zeros((o.nyp, o.nxp), dtype=bool)
    bnd[[0, -1], :] = True
    if not periodic:
        bnd[:, [0, -1]] = True
    np.testing.assert_array_equal(V[~bnd], U.reshape(o.nyp, o.nxp)[~bnd])
    X, Y = o.node_coords()
    for (xi, eta), v in zip(zip(X[bnd], Y[bnd]), V[bnd]):
        m = o.map(xi, eta)
        want = 0.0 if periodic else math.exp(m[0] + m[1] + t)
        assert v == pytest.approx(want, rel=1e-15, abs=0.0)
