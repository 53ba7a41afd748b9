"""Convergence, analytical-solution and paper-table pins for the oracle:
Bessel cross products of eq. (Annulus_AS) against scipy, the paper's
normalisation B_{1,m}, observed order under refinement for a manufactured
solution and for exact annulus eigenmodes, the full-domain solver, and the
printed error tables of Section 4 (tests/golden/paper_tables.json)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.special as sp

from paper_2405_08764_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


@pytest.mark.parametrize("k,ra,rb", [(1, 1.0, 2.0), (2, 1.0, 2.0), (3, 0.7, 2.6), (4, 1.0, 2.0)])
def test_bessel_roots_match_scipy(orc, k, ra, rb):
    f = lambda mu: sp.jv(k, mu * ra) * sp.yv(k, mu * rb) - sp.yv(k, mu * ra) * sp.jv(k, mu * rb)  # noqa: E731
    grid = np.linspace(0.05, 40, 20000)
    vals = f(grid)
    roots = [so.brentq(f, grid[q], grid[q + 1], xtol=1e-15)
             for q in range(len(grid) - 1) if vals[q] * vals[q + 1] < 0][:3]
    for which, want in enumerate(roots, start=1):
        assert abs(orc.bessel_root(k, ra, rb, which) - want) < 1e-11 * want


@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_bessel_norm_equals_paper_B1m(orc, m):
    """Eq. (Annulus_AS): 1 / int_1^2 r Z_1(mu r)^2 dr = (pi^2/2) B_{1,m},
    B_{1,m} = mu^2 J_1(2mu)^2 / (J_1(mu)^2 - J_1(2mu)^2)."""
    mu = orc.bessel_root(1, 1.0, 2.0, m)
    B = mu ** 2 * sp.jv(1, 2 * mu) ** 2 / (sp.jv(1, mu) ** 2 - sp.jv(1, 2 * mu) ** 2)
    np.testing.assert_allclose(1.0 / orc.bessel_norm(mu, 1.0, 2.0, 4000), math.pi ** 2 / 2 * B, rtol=1e-9)


def test_annulus_series_reproduces_initial_data(orc):
    for r in (1.1, 1.37, 1.5, 1.81, 1.95):
        for th in (0.3, 1.9, 4.4):
            want = (r - 1) * (2 - r) * math.sin(th)
            assert abs(orc.annulus_series(1, 2, r, th, 0.0, 40) - want) < 2e-5


def test_annulus_initial_data_of_section_4_2(orc):
    """The Section 4.2 initial field at the macro nodes of a stretched annulus:
    (r - 1)(2 - r) sin(theta), with r and theta of each node's physical point."""
    p = W.c3_annulus(n_r=9, n_theta=16, m=5)
    o = orc.Oracle(p)
    U = o.init_field(kind="annulus_poly", params=[1.0, 2.0])
    X, Y = o.node_coords()
    for (xi, eta), u in zip(zip(X.ravel(), Y.ravel()), U):
        m = o.map(xi, eta)
        r, th = math.hypot(m[0], m[1]), math.atan2(m[1], m[0])
        assert abs(u - (r - 1.0) * (2.0 - r) * math.sin(th)) <= 1e-14


@pytest.mark.parametrize("d0", [1.0, 0.4])
def test_bessel_mode_field_solves_the_heat_equation(orc, d0):
    """The eigenmode initial field decays as exp(-d0 mu^2 t) and satisfies
    u_t = d0 Laplacian u for the diffusivity d0 (checked by finite differences
    in r, theta)."""
    p = W.c3_annulus(n_r=15, n_theta=24, m=5)
    p["d_aff"] = (d0, 0.0, 0.0)
    o = orc.Oracle(p)
    U1, U2 = o.init_field(t=0.01), o.init_field(t=0.01 + 1e-6)
    dUdt = (U2 - U1) / 1e-6
    mus = [orc.bessel_root(k, 1.0, 2.0, 1) for k in range(1, 5)]
    amps = p["init_p"][3:]
    X, Y = o.node_coords()
    for (th, eta), ut in list(zip(zip(X.ravel(), Y.ravel()), dUdt))[::17]:
        r = o.map(th, eta)
        rr = math.hypot(r[0], r[1])
        want = sum(-d0 * mu * mu * a * orc.bessel_Z(k, mu, 1.0, rr) * math.cos(k * th)
                   * math.exp(-d0 * mu * mu * 0.01) for k, (mu, a) in enumerate(zip(mus, amps), start=1))
        assert abs(ut - want) < 1e-4 * (1 + abs(want))
        # and the mode satisfies Bessel's equation: Z'' + Z'/r + (mu^2 - k^2/r^2) Z = 0
        for k, mu in enumerate(mus, start=1):
            h = 1e-4
            z = lambda x: orc.bessel_Z(k, mu, 1.0, x)  # noqa: E731
            z1 = (z(rr + h) - z(rr - h)) / (2 * h)
            z2 = (z(rr + h) - 2 * z(rr) + z(rr - h)) / h ** 2
            assert abs(z2 + z1 / rr + (mu * mu - k * k / rr ** 2) * z(rr)) < 1e-4 * mu * mu


def _manufactured_error(orc, n, conv):
    p = W.c1_manufactured(n=n, n_macro=50 * (n // 8) ** 2, dt_macro=0.01 / (n // 8) ** 2)
    p["conv"] = conv
    o = orc.Oracle(p)
    U = o.step(o.init_field(), 0.0, p["dt_macro"], p["n_macro"])
    X, Y = o.node_coords()
    ex = math.exp(-0.5) * np.sin(math.pi * X) * np.sin(math.pi * Y)
    return np.linalg.norm(U - ex.ravel()) / np.linalg.norm(ex)


def test_manufactured_solution_second_order_with_central_micro_convection(orc):
    """Manufactured u = exp(-t) sin(pi x) sin(pi y) with the source of the
    5-config benchmark; Delta t ~ Delta^2, h / Delta fixed: observed order >= 1.9."""
    e = [_manufactured_error(orc, n, "central") for n in (8, 16, 32)]
    orders = [math.log2(e[q] / e[q + 1]) for q in range(2)]
    assert min(orders) > 1.9, (e, orders)


def test_manufactured_solution_upwind_converges(orc):
    """With the 2-point upwind micro difference (Section 4.1.1) the O(delta)
    upwind error takes over on fine grids; the error still falls monotonically
    with order >= 1 and the coarse-grid error is below 2.5%."""
    e = [_manufactured_error(orc, n, "upwind") for n in (8, 16, 32)]
    assert e[0] < 0.025 and all(math.log2(e[q] / e[q + 1]) > 0.95 for q in range(2)), e


def test_annulus_eigenmodes_second_order(orc):
    """Two exact eigenmodes of the stretched annulus (generalising eq. (Annulus_AS));
    periodic xi, stretched radial map: observed order >= 1.9."""
    errs = []
    for nt, nr in ((16, 8), (32, 16), (64, 32)):
        p = W.base(n_xi=nt, n_eta=nr, periodic_xi=1, box=(0, 2 * math.pi, 0, 1), map="polar",
                   map_p=(1, 2, 1.5, 0), m_xi=9, m_eta=9, conv="central", init="bessel",
                   init_p=[2.0, 1.0, 2.0, 1.0, 0.7])
        o = orc.Oracle(p)
        dtm = o.dt_macro()
        n = int(math.ceil(0.02 / dtm))
        U = o.step(o.init_field(t=0.0), 0.0, 0.02 / n, n)
        ex = o.init_field(t=0.02)
        errs.append(np.linalg.norm(U - ex) / np.linalg.norm(ex))
    orders = [math.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert min(orders) > 1.9, (errs, orders)


def test_full_domain_solver_converges_to_manufactured_solution(orc):
    errs = []
    for refine in (2, 4):
        p = W.c1_manufactured(n=8)
        p["conv"] = "central"
        o = orc.Oracle(p)
        ny, nx = o.full_domain_shape(refine)
        xi = np.linspace(0, 1, nx)
        X, Y = np.meshgrid(xi, np.linspace(0, 1, ny))
        u = (np.sin(math.pi * X) * np.sin(math.pi * Y)).ravel()
        h = 1.0 / (8 * refine)
        dt = 0.2 * h * h / 0.05
        n = int(math.ceil(0.1 / dt))
        u = o.full_domain(u, refine, 0.0, 0.1 / n, n)
        ex = (math.exp(-0.1) * np.sin(math.pi * X) * np.sin(math.pi * Y)).ravel()
        errs.append(np.abs(u - ex).max())
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_full_domain_step_is_exact_on_quadratics(orc):
    """Central differences are exact on quadratics, so one forward-Euler step
    of the full-domain solver from u = q(x, y) (identity map, constant tensor
    with a cross term, constant v, reaction, source s(t) G at the step's start
    time) is q + dt (L q + s(t0) G) at every interior node, with L q in closed
    form; the boundary nodes take the exact solution at t0 + dt."""
    a11, a12, a22, d, v1, v2, f0 = 1.0, 0.3, 0.7, 0.05, 0.8, -0.6, 0.25
    sp = (0.4, -1.0, 0.5)
    p = W.base(n_xi=6, n_eta=5, conv="central", M=(a11, a12, a22), d_aff=(d, 0.0, 0.0), va=(v1, 0.0, 0.0),
               vb=(v2, 0.0, 0.0), f0=f0, src="exp_linear", src_p=sp, time="exp", tc=1.0, sol="exp_xyt")
    o = orc.Oracle(p)
    refine = 2
    ny, nx = o.full_domain_shape(refine)
    X, Y = np.meshgrid(np.linspace(0, 1, nx), np.linspace(0, 1, ny))
    q00, q10, q01, q20, q11, q02 = 0.3, -0.7, 0.4, 1.1, -0.9, 0.6
    q = q00 + q10 * X + q01 * Y + q20 * X * X + q11 * X * Y + q02 * Y * Y
    t0, dt = 0.2, 1e-4
    got = o.full_domain(q.ravel(), refine, t0, dt, 1).reshape(ny, nx)
    Lq = (d * a11 * 2 * q20 + 2 * d * a12 * q11 + d * a22 * 2 * q02
          - v1 * (q10 + 2 * q20 * X + q11 * Y) - v2 * (q01 + q11 * X + 2 * q02 * Y) + f0 * q)
    G = (sp[0] + sp[1] * X + sp[2] * Y) * np.exp(X + Y)
    want = q + dt * (Lq + math.exp(t0) * G)
    np.testing.assert_allclose(got[1:-1, 1:-1], want[1:-1, 1:-1], rtol=0, atol=1e-12)
    bnd = np.ones_like(q, dtype=bool)
    bnd[1:-1, 1:-1] = False
    np.testing.assert_allclose(got[bnd], np.exp(X + Y + t0 + dt)[bnd], rtol=1e-14)


def _max_pct_error(orc, p, n_steps, t_end=1.0, chunks=20):
    o = orc.Oracle(p)
    U = o.init_field()
    X, Y = o.node_coords()
    xy = np.array([o.map(a, b)[:2] for a, b in zip(X.ravel(), Y.ravel())])
    worst = 0.0
    for c in range(chunks):
        U = o.step(U, c * t_end / chunks, t_end / n_steps, n_steps // chunks)
        ex = np.exp(xy[:, 0] + xy[:, 1] + (c + 1) * t_end / chunks)
        worst = max(worst, 100 * np.max(np.abs(U - ex) / ex))
    return worst


@pytest.mark.parametrize("variable_d,table", [(False, "table2_constant_diffusivity"),
                                              (True, "table4_variable_diffusivity")])
def test_paper_tables_2_and_4(orc, variable_d, table):
    """Section 4.1 rerun with forward-Euler bursts at the tables' macro settings:
    max % error within a factor 1.5 of the printed value, lambda = 0.1 best."""
    g = GOLD[table]
    want = g["columns"][0]["max_percent_error"][:3]
    got = [_max_pct_error(orc, W.paper_cdr(variable_d, lam=lam), 2000) for lam in g["lambda"][:3]]
    for mine, paper in zip(got, want):
        assert paper / 1.5 < mine < paper * 1.5, (got, want)
    assert got[1] < got[0] and got[1] < got[2]


def _printed_unit(v):
    """one unit in the last of the three printed significant digits"""
    return 10.0 ** (math.floor(math.log10(abs(v))) - 2)


@pytest.mark.parametrize("variable_d,table,lams", [(False, "table2_constant_diffusivity", (0.0, 0.1, 0.3, 0.6)),
                                                   (True, "table4_variable_diffusivity", (0.0, 0.2, 0.5))])
def test_paper_tables_reproduced_with_adi_bursts(orc, variable_d, table, lams):
    """Section 4.1 at the paper's own micro settings (ADI, n_t = 2, tau = 1e-6,
    h = 1e-3, n = 10) and the printed restriction reference: the 10 x 10,
    N_t = 2000 column of Tables 2 and 4 to within one unit of the last printed
    digit.  The tables' maximum is taken over the macro nodes at t = 1 (the
    maximum over earlier times as well differs in the third digit at
    lambda = 0.1)."""
    g = GOLD[table]
    col = g["columns"][0]
    for lam in lams:
        want = col["max_percent_error"][g["lambda"].index(lam)]
        p = W.paper_cdr_adi(variable_d, lam, col["n"], col["n_t"])
        got = _max_pct_error(orc, p, col["n_t"], chunks=1)
        assert abs(got - want) <= _printed_unit(want), (lam, got, want)


def test_paper_table7_annulus(orc):
    """Section 4.2 at the paper's patch settings (h = 1e-3, n = 20), first column
    of Table 7: max relative error at t = 0.05 within a factor 3 of 1.40e-3."""
    g = GOLD["table7_annulus"]
    p = W.paper_annulus(16, 10, m=21)
    p["h_ratio_xi"] = 1e-3 / (2 * math.pi / 16)
    p["h_ratio_eta"] = 1e-3 / 0.1
    o = orc.Oracle(p)
    U = o.step(o.init_field(), 0.0, 0.2 / 500, 125)
    X, Y = o.node_coords()
    ua = np.array([orc.annulus_series(1, 2, r, th, 0.05, 40) for th, r in zip(X.ravel(), Y.ravel())])
    err = np.abs(U - ua).max() / np.abs(ua).max()
    assert g["max_relative_error"][0] / 3 < err < 3 * g["max_relative_error"][0], err
