"""Pins for the oracle's maps and transformed coefficients (Section 2, eq.
(Computational_Problem)) against what the paper and the mathematics fix:
the worked coefficient sets of Section 4, the identity-map special case, and the
invariant that the transformed operator equals the physical one."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W

RNG = np.random.default_rng(1234)


def _pts(n, lo=0.02, hi=0.98):
    return RNG.uniform(lo, hi, size=(n, 2))


@pytest.mark.parametrize("lam", [0.0, 0.1, 0.3, 0.6])
def test_sine_map_constant_diffusivity_matches_eq_P1_C(orc, lam):
    """Section 4.1.1, eq. (P1_C): alpha, gamma = 1/(1 + lambda cos)^2, beta = 0,
    nu = 10 x / x_xi - lambda pi sin(pi xi) / x_xi^3 (likewise omega), phi = 0."""
    o = orc.Oracle(W.paper_cdr(False, lam=lam))
    for xi, eta in _pts(25):
        c = o.coeffs(xi, eta)
        X = xi + lam / math.pi * math.sin(math.pi * xi)
        Y = eta + lam / math.pi * math.sin(math.pi * eta)
        Jx = 1 + lam * math.cos(math.pi * xi)
        Jy = 1 + lam * math.cos(math.pi * eta)
        want = [1 / Jx ** 2, 0.0, 1 / Jy ** 2,
                10 * X / Jx - lam * math.pi * math.sin(math.pi * xi) / Jx ** 3,
                10 * Y / Jy - lam * math.pi * math.sin(math.pi * eta) / Jy ** 3, 0.0]
        np.testing.assert_allclose(c[:6], want, rtol=1e-13, atol=1e-13)
        # g of eq. (P1_C) without the time factor exp(t)
        np.testing.assert_allclose(c[6], (10 * X + 10 * Y - 1) * math.exp(X + Y), rtol=1e-13)


@pytest.mark.parametrize("lam", [0.0, 0.1, 0.4])
def test_sine_map_variable_diffusivity_matches_eq_P1_C_Vari_Diff(orc, lam):
    """Section 4.1.2, eq. (P1_C_Vari_Diff): D = 1 + x, v = (1 + 10x, 10y)."""
    o = orc.Oracle(W.paper_cdr(True, lam=lam))
    for xi, eta in _pts(25):
        c = o.coeffs(xi, eta)
        X = xi + lam / math.pi * math.sin(math.pi * xi)
        Y = eta + lam / math.pi * math.sin(math.pi * eta)
        Jx = 1 + lam * math.cos(math.pi * xi)
        Jy = 1 + lam * math.cos(math.pi * eta)
        want = [(1 + X) / Jx ** 2, 0.0, (1 + X) / Jy ** 2,
                10 * X / Jx - lam * math.pi * math.sin(math.pi * xi) * (1 + X) / Jx ** 3,
                10 * Y / Jy - lam * math.pi * math.sin(math.pi * eta) * (1 + X) / Jy ** 3, 0.0]
        np.testing.assert_allclose(c[:6], want, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(c[6], (8 * X + 10 * Y - 1) * math.exp(X + Y), rtol=1e-13)


def test_polar_map_matches_eq_Ann_Diff_Computational(orc):
    """Section 4.2, eq. (Ann_Diff_Computational): alpha = 1/eta^2, gamma = 1,
    omega = -1/eta, everything else zero."""
    o = orc.Oracle(W.paper_annulus())
    for th, r in RNG.uniform([0, 1.0], [2 * math.pi, 2.0], size=(25, 2)):
        c = o.coeffs(th, r)
        np.testing.assert_allclose(c[:6], [1 / r ** 2, 0, 1, 0, -1 / r, 0], rtol=1e-13, atol=1e-14)


def test_identity_map_reduces_to_cartesian_operator(orc):
    """Special case: with x = xi, y = eta the operator of eq. (1) expanded by hand,
    alpha = K11, beta = 2 K12, gamma = K22, nu = v1 - dK11/dx - dK12/dy,
    omega = v2 - dK12/dx - dK22/dy, phi = f - div v."""
    p = W.base(M=(1.0, 0.3, 0.7), d_aff=(0.5, 0.2, -0.1), d_sin=(0.1, 1.0),
               va=(0.3, 1.1, -0.4), vb=(-0.2, 0.5, 0.9), f0=0.7)
    o = orc.Oracle(p)
    for x, y in _pts(20):
        d = 0.5 + 0.2 * x - 0.1 * y + 0.1 * math.sin(2 * math.pi * x) * math.sin(2 * math.pi * y)
        ddx = 0.2 + 0.1 * 2 * math.pi * math.cos(2 * math.pi * x) * math.sin(2 * math.pi * y)
        ddy = -0.1 + 0.1 * 2 * math.pi * math.sin(2 * math.pi * x) * math.cos(2 * math.pi * y)
        v1 = 0.3 + 1.1 * x - 0.4 * y
        v2 = -0.2 + 0.5 * x + 0.9 * y
        want = [d * 1.0, 2 * d * 0.3, d * 0.7,
                v1 - ddx * 1.0 - ddy * 0.3, v2 - ddx * 0.3 - ddy * 0.7, 0.7 - (1.1 + 0.9)]
        np.testing.assert_allclose(o.coeffs(x, y)[:6], want, rtol=1e-13, atol=1e-14)


def _fd_derivs(f, a, b, h):
    """4th-order central differences of f(a, b): f_a, f_b, f_aa, f_ab, f_bb."""
    fa = (-f(a + 2 * h, b) + 8 * f(a + h, b) - 8 * f(a - h, b) + f(a - 2 * h, b)) / (12 * h)
    fb = (-f(a, b + 2 * h) + 8 * f(a, b + h) - 8 * f(a, b - h) + f(a, b - 2 * h)) / (12 * h)
    faa = (-f(a + 2 * h, b) + 16 * f(a + h, b) - 30 * f(a, b) + 16 * f(a - h, b) - f(a - 2 * h, b)) / (12 * h * h)
    fbb = (-f(a, b + 2 * h) + 16 * f(a, b + h) - 30 * f(a, b) + 16 * f(a, b - h) - f(a, b - 2 * h)) / (12 * h * h)

    def fb_at(aa):
        return (-f(aa, b + 2 * h) + 8 * f(aa, b + h) - 8 * f(aa, b - h) + f(aa, b - 2 * h)) / (12 * h)
    fab = (-fb_at(a + 2 * h) + 8 * fb_at(a + h) - 8 * fb_at(a - h) + fb_at(a - 2 * h)) / (12 * h)
    return fa, fb, faa, fab, fbb


MAP_CASES = [
    W.base(map="sine", map_p=(0.35, 0, 0, 0)),
    W.base(map="tanh", map_p=(3.0, 2.0, 0, 0)),
    W.base(map="polar", map_p=(1.0, 2.0, 1.5, 0), periodic_xi=1, box=(0, 2 * math.pi, 0, 1)),
    W.base(map="polar", map_p=(0.7, 2.4, 0.0, 0), periodic_xi=1, box=(0, 2 * math.pi, 0, 1)),
]


@pytest.mark.parametrize("case", range(len(MAP_CASES)))
def test_map_derivatives_by_finite_differences(orc, case):
    o = orc.Oracle(MAP_CASES[case])
    for xi, eta in _pts(6, 0.2, 0.8):
        m = o.map(xi, eta)
        for comp, idx in ((0, (2, 3, 6, 7, 8)), (1, (4, 5, 9, 10, 11))):
            fd = _fd_derivs(lambda a, b: o.map(a, b)[comp], xi, eta, 1e-3)
            np.testing.assert_allclose([m[k] for k in idx], fd, rtol=1e-7, atol=1e-7)


def _hetero(prob):
    prob = dict(prob)
    prob.update(M=(1.0, 0.35, 0.6), d_aff=(0.8, 0.3, -0.2), d_sin=(0.2, 1.0),
                va=(0.4, 1.2, -0.5), vb=(-0.3, 0.6, 0.8), f0=0.9,
                four=dict(c=[0.05, -0.04, 0.03], phi=[0.3, 1.1, 2.0], ra=0.5, rb=3.0))
    return prob


def test_physical_coefficient_gradients_by_finite_differences(orc):
    o = orc.Oracle(_hetero(MAP_CASES[2]))
    for x, y in RNG.uniform(0.6, 1.4, size=(6, 2)):
        ph = o.physical(x, y)
        for c in range(3):
            fd = _fd_derivs(lambda a, b: o.physical(a, b)[c], x, y, 1e-3)
            np.testing.assert_allclose([ph[3 + c], ph[6 + c]], fd[:2], rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("case", range(len(MAP_CASES)))
def test_transformed_operator_equals_physical_operator(orc, case):
    """Invariant: for any smooth u, alpha u_xixi + beta u_xieta + gamma u_etaeta
    - nu u_xi - omega u_eta + phi u computed in (xi, eta) equals div(K grad u)
    - div(v u) + f u computed in (x, y).  Pins every term of the transformed
    operator (signs, cross term, Jacobian) for every map, with tensor K."""
    o = orc.Oracle(_hetero(MAP_CASES[case]))

    def u(x, y):
        return math.sin(1.3 * x + 0.4) * math.cos(0.9 * y - 0.2) + 0.3 * x * x * y

    def ux(x, y):
        return 1.3 * math.cos(1.3 * x + 0.4) * math.cos(0.9 * y - 0.2) + 0.6 * x * y

    def uy(x, y):
        return -0.9 * math.sin(1.3 * x + 0.4) * math.sin(0.9 * y - 0.2) + 0.3 * x * x

    def uxx(x, y):
        return -1.69 * math.sin(1.3 * x + 0.4) * math.cos(0.9 * y - 0.2) + 0.6 * y

    def uyy(x, y):
        return -0.81 * math.sin(1.3 * x + 0.4) * math.cos(0.9 * y - 0.2)

    def uxy(x, y):
        return -1.17 * math.cos(1.3 * x + 0.4) * math.sin(0.9 * y - 0.2) + 0.6 * x

    for xi, eta in _pts(6, 0.2, 0.8):
        m = o.map(xi, eta)
        x, y = m[0], m[1]
        ph = o.physical(x, y)
        K11, K12, K22 = ph[0:3]
        dK11x, dK12x, dK22x, dK11y, dK12y, dK22y = ph[3:9]
        v1, v2, divv, f = ph[9:13]
        phys = (K11 * uxx(x, y) + 2 * K12 * uxy(x, y) + K22 * uyy(x, y)
                + (dK11x + dK12y) * ux(x, y) + (dK12x + dK22y) * uy(x, y)
                - (v1 * ux(x, y) + v2 * uy(x, y)) - divv * u(x, y) + f * u(x, y))
        comp_u = lambda a, b: u(*o.map(a, b)[:2])  # noqa: E731
        fa, fb, faa, fab, fbb = _fd_derivs(comp_u, xi, eta, 1e-3)
        c = o.coeffs(xi, eta)
        comp = c[0] * faa + c[1] * fab + c[2] * fbb - c[3] * fa - c[4] * fb + c[5] * u(x, y)
        assert abs(comp - phys) <= 1e-6 * (1 + abs(phys)), (case, xi, eta, comp, phys)


def _d1(f, z, h):
    """fourth-order central difference"""
    return (8.0 * (f(z + h) - f(z - h)) - (f(z + 2 * h) - f(z - 2 * h))) / (12.0 * h)


def test_manufactured_source_satisfies_the_pde(orc):
    """u = exp(-t) sin(pi x) sin(pi y) solves u_t = div(K grad u - v u) + f u +
    s(t) G for the manufactured source with a constant tensor K (cross term),
    an affine v with non-zero divergence and f != 0: the residual, with every
    derivative of u and of the flux taken by fourth-order central differences,
    vanishes at random points."""
    M, d, va, vb, f0 = (0.7, 0.2, 1.1), 0.05, (0.5, 0.3, 0.1), (-0.4, 0.2, -0.3), 0.3
    o = orc.Oracle(W.base(M=M, d_aff=(d, 0.0, 0.0), va=va, vb=vb, f0=f0, src="mms_sinprod", time="exp",
                          tc=-1.0))
    K = d * np.array([[M[0], M[1]], [M[1], M[2]]])
    h, t = 1e-3, 0.37

    def u(x, y, s):
        return math.exp(-s) * math.sin(math.pi * x) * math.sin(math.pi * y)

    def flux(x, y):
        ux = _d1(lambda z: u(z, y, t), x, h)
        uy = _d1(lambda z: u(x, z, t), y, h)
        v1 = va[0] + va[1] * x + va[2] * y
        v2 = vb[0] + vb[1] * x + vb[2] * y
        uu = u(x, y, t)
        return K[0, 0] * ux + K[0, 1] * uy - v1 * uu, K[1, 0] * ux + K[1, 1] * uy - v2 * uu

    for x, y in _pts(20):
        div = _d1(lambda z: flux(z, y)[0], x, h) + _d1(lambda z: flux(x, z)[1], y, h)
        g = _d1(lambda s: u(x, y, s), t, h) - div - f0 * u(x, y, t)
        G = o.coeffs(x, y)[6]                      # identity map: computational = physical
        assert abs(o.time_factor(t) * G - g) <= 1e-8 * (1.0 + abs(g)), (x, y, o.time_factor(t) * G, g)


def test_manufactured_exact_solution_solves_the_problem_with_its_source(orc):
    """The oracle's exact solution of the manufactured problem (Dirichlet and
    initial data) and its source belong together: the residual of
    u_t = div(K grad u - v u) + f u + s(t) G with u = the oracle's exact
    solution, derivatives by fourth-order central differences, vanishes."""
    M, d, va, vb, f0 = (0.9, -0.15, 0.6), 0.07, (0.2, -0.4, 0.3), (0.5, 0.1, 0.2), -0.2
    o = orc.Oracle(W.base(M=M, d_aff=(d, 0.0, 0.0), va=va, vb=vb, f0=f0, src="mms_sinprod", time="exp",
                          tc=-1.0, sol="sinprod_decay"))
    K = d * np.array([[M[0], M[1]], [M[1], M[2]]])
    h = 1e-3
    for (x, y), t in zip(_pts(12), np.linspace(0.1, 0.9, 12)):
        def flux(a, b):
            ux = _d1(lambda z: o.exact(z, b, t), a, h)
            uy = _d1(lambda z: o.exact(a, z, t), b, h)
            uu = o.exact(a, b, t)
            v1 = va[0] + va[1] * a + va[2] * b
            v2 = vb[0] + vb[1] * a + vb[2] * b
            return K[0, 0] * ux + K[0, 1] * uy - v1 * uu, K[1, 0] * ux + K[1, 1] * uy - v2 * uu
        div = _d1(lambda z: flux(z, y)[0], x, h) + _d1(lambda z: flux(x, z)[1], y, h)
        res = _d1(lambda s: o.exact(x, y, s), t, h) - div - f0 * o.exact(x, y, t) - o.time_factor(t) * o.coeffs(x, y)[6]
        assert abs(res) <= 1e-8, (x, y, t, res)


def test_bump_initial_field(orc):
    """The batch workload's initial field: sin(pi z_xi) sin(pi z_eta) with z the
    position in the computational box, or (1 + cos(xi)/2) sin(pi z_eta) when xi
    is periodic."""
    for p in (W.base(n_xi=7, n_eta=5, box=(0.0, 2.0, -1.0, 1.0), init="bump"),
              W.base(n_xi=12, n_eta=5, periodic_xi=1, map="polar", map_p=(1.0, 2.0, 0, 0),
                     box=(0.0, 2.0 * math.pi, 0.0, 1.0), init="bump")):
        o = orc.Oracle(p)
        U = o.init_field().reshape(o.nyp, o.nxp)
        X, Y = o.node_coords()
        x0, x1, y0, y1 = p["box"]
        zy = (Y - y0) / (y1 - y0)
        fx = (1.0 + 0.5 * np.cos(X)) if p["periodic_xi"] else np.sin(math.pi * (X - x0) / (x1 - x0))
        np.testing.assert_allclose(U, fx * np.sin(math.pi * zy), rtol=0, atol=1e-15)


def test_workload_fields_match_their_definitions(orc):
    """The synthetic fields as documented for the workloads: the annulus
    diffusivity d = 1 + sum_k c_k cos(k theta + phi_k) cos(k pi rho),
    rho = (r - 1) / (2 - 1), and the Gaussian source factor exp(-(x^2 + y^2))."""
    p = W.c5_surrogate_field(n_r=7, n_theta=16)
    o = orc.Oracle(p)
    c, ph = p["four"]["c"], p["four"]["phi"]
    rng = np.random.default_rng(9)
    for r, th in zip(rng.uniform(1.0, 2.0, 20), rng.uniform(-math.pi, math.pi, 20)):
        x, y = r * math.cos(th), r * math.sin(th)
        want = 1.0 + sum(c[k - 1] * math.cos(k * th + ph[k - 1]) * math.cos(k * math.pi * (r - 1.0))
                         for k in (1, 2, 3))
        assert o.physical(x, y)[0] == pytest.approx(want, rel=1e-14)
    q = W.base(n_xi=5, n_eta=5, src="gauss_patch", src_amp=np.ones(16), time="sin", tc=math.pi)
    og = orc.Oracle(q)
    for x, y in _pts(10):
        assert og.coeffs(x, y)[6] == pytest.approx(math.exp(-(x * x + y * y)), rel=1e-14)
