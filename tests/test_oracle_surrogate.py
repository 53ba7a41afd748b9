"""Pins of the surrogate oracle (oracle/surrogate.py) against facts that do not
come from it: central finite differences for the backward pass, the odd-part
identity of GELU, exact discrete derivatives of polynomials for the stencil
basis, scale invariance, closed-form metric terms for the identity map, the
summation-by-parts K-independence of the patch scheme, and the plain scheme
as the all-fallback limit of the surrogate step."""
import math

import numpy as np
import pytest

from oracle import Oracle
from oracle import surrogate as S
from paper_2405_08764_gb300 import workloads as W


def test_gelu_odd_part_and_limits():
    x = np.linspace(-9.0, 9.0, 1001)
    # tanh is odd, so g(x) - g(-x) = x exactly for the tanh form
    np.testing.assert_allclose(S.gelu(x) - S.gelu(-x), x, rtol=0, atol=4e-15)
    assert S.gelu(0.0) == 0.0
    assert abs(S.gelu(30.0) - 30.0) < 1e-12 and abs(S.gelu(-30.0)) < 1e-12
    h = 1e-6
    fd = (S.gelu(x + h) - S.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(S.gelu_grad(x), fd, rtol=0, atol=1e-8)
    # the tanh form stays within 1e-3 of x * Phi(x)
    from math import erf
    exact = np.array([0.5 * v * (1 + erf(v / math.sqrt(2))) for v in x])
    assert np.abs(S.gelu(x) - exact).max() < 1e-3


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 0.0, 3.0e38])
    want = np.array([1.0, 1.0, 1.0 + 4 * 2 ** -8, 1.0, -2.5, 0.0, 1.765625 * 2.0 ** 127])
    got = S.bf16(vals)
    np.testing.assert_array_equal(got[:6], want[:6])      # ties go to even
    assert got[6] == want[6]
    r = np.random.default_rng(0).normal(size=10000) * 10.0 ** np.random.default_rng(1).uniform(-20, 20, 10000)
    rel = np.abs(S.bf16(r) - r.astype(np.float32)) / np.abs(r.astype(np.float32))
    assert rel.max() <= 2.0 ** -8      # 8 significant bits: unit roundoff 2^-8


def _theta(seed=3, scale=1.0):
    th = S.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    p = S.unflatten(th)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.normal(size=p[k].shape)
    p["b4"] = np.array([0.05])
    p["W1"][:, S.N_IN:] = 0.0
    return S.flatten(p) * scale


def test_backward_matches_central_differences():
    rng = np.random.default_rng(7)
    th = _theta()
    X = rng.normal(size=(9, S.N_IN))
    t = rng.normal(size=9)
    g = S.gradient(th, X, t)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in S.SHAPES])
    idx = []
    for k in range(len(S.SHAPES)):          # components of every tensor
        idx += list(rng.integers(offs[k], offs[k + 1], 12))
    idx += list(range(offs[0] + S.N_IN, offs[0] + S.N_IN + 3))   # padding columns: zero gradient
    for i in idx:
        h = 1e-6 * max(1.0, abs(th[i]))
        a, b = th.copy(), th.copy()
        a[i] += h
        b[i] -= h
        fd = (S.loss(a, X, t) - S.loss(b, X, t)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, g[i], fd)
    assert np.all(S.unflatten(g)["W1"][:, S.N_IN:] == 0.0)


def test_forward_special_weights():
    p = S.unflatten(np.zeros(S.N_PARAM))
    p["b3"] = np.linspace(-2, 2, S.WIDTH)
    p["w4"] = np.linspace(1, 3, S.WIDTH)
    p["b4"] = np.array([0.5])
    X = np.random.default_rng(0).normal(size=(4, S.N_IN))
    y, _ = S.forward(S.flatten(p), X)
    want = float(S.gelu(p["b3"]) @ p["w4"] + 0.5)
    np.testing.assert_allclose(y, want, rtol=1e-15)


def test_adam_first_step_closed_form():
    g = np.array([2.0, -0.5, 0.0, 1e-3])
    th = np.ones(4)
    th1, m, v = S.adam(th, g, np.zeros(4), np.zeros(4), 1, 0.01)
    # with zero moments the bias-corrected step is lr * g / (|g| + eps)
    np.testing.assert_allclose(th1, 1.0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def _poly_stencil(f, dx, dy):
    q, p = np.meshgrid(np.arange(-2, 3), np.arange(-2, 3), indexing="ij")
    return f(0.3 + p * dx, -0.2 + q * dy)[None]


def test_stencil_basis_gives_exact_differences_of_polynomials():
    dx, dy = 0.1, 0.05
    # cubic in xi times quadratic in eta: every basis term has a closed form
    f = lambda x, y: (1 + 2 * x - x ** 2 + 0.5 * x ** 3) * (3 - y + 4 * y ** 2)
    st = _poly_stencil(f, dx, dy)
    a = S.basis_1d(st)
    D = np.swapaxes(S.basis_1d(np.swapaxes(a, 1, 2)), 1, 2).reshape(25)
    x0, y0 = 0.3, -0.2
    fx = [1 + 2 * x0 - x0 ** 2 + 0.5 * x0 ** 3, 2 - 2 * x0 + 1.5 * x0 ** 2, -2 + 3 * x0, 3.0, 0.0]
    gy = [3 - y0 + 4 * y0 ** 2, -1 + 8 * y0, 8.0, 0.0, 0.0]
    # central first difference of a cubic: u' dx + u''' dx^3 / 6
    dfx = [fx[0], fx[1] * dx + fx[3] * dx ** 3 / 6, fx[2] * dx ** 2, fx[3] * dx ** 3, 0.0]
    dgy = [gy[0], gy[1] * dy, gy[2] * dy ** 2, 0.0, 0.0]
    want = np.array([dfx[pp] * dgy[qq] for qq in range(5) for pp in range(5)])
    np.testing.assert_allclose(D, want, rtol=0, atol=1e-12)
    x, s = S.stencil_features(st)
    np.testing.assert_allclose(s[0], np.abs(want[1:]).max(), rtol=1e-13)
    np.testing.assert_allclose(x[0, 1:], want[1:] / s[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(x[0, 0], want[0] / (abs(want[0]) + s[0]), rtol=1e-14)


def test_stencil_basis_is_invertible_and_scale_invariant():
    E = np.eye(25).reshape(25, 5, 5)
    Mx = np.stack([np.swapaxes(S.basis_1d(np.swapaxes(S.basis_1d(e[None]), 1, 2)), 1, 2).reshape(25) for e in E])
    assert np.linalg.matrix_rank(Mx) == 25 and np.linalg.cond(Mx) < 1e3
    st = np.random.default_rng(4).normal(size=(50, 5, 5))
    x, s = S.stencil_features(st)
    x2, s2 = S.stencil_features(3.7 * st)
    np.testing.assert_allclose(x2, x, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(s2, 3.7 * s, rtol=1e-15)
    x3, _ = S.stencil_features(-st)
    np.testing.assert_allclose(x3, -x, rtol=1e-13, atol=1e-15)
    z, sz = S.stencil_features(np.zeros((2, 5, 5)))
    assert np.all(z == 0) and np.all(sz == 0)


def test_stencils_wrap_in_xi_and_clamp_in_eta():
    p = W.c5_surrogate_field(n_r=6, n_theta=10, m=5)
    o = Oracle(p)
    U = np.arange(o.n_macro, dtype=np.float64)
    st = S.stencils(o, U)
    I, J = o.patch_nodes()
    for k in (0, 9, 10, 44):
        for q in range(-2, 3):
            for pp in range(-2, 3):
                r = min(max(J[k] + q, 0), 6)
                c = (I[k] + pp) % 10
                assert st[k, q + 2, pp + 2] == r * 10 + c


def test_static_features_identity_map_closed_form():
    d, v1, v2, f = 0.05, 1.0, -0.5, 0.0
    p = W.base(n_xi=6, n_eta=5, M=(1.0, 0.0, 1.0), d_aff=(d, 0.0, 0.0), va=(v1, 0.0, 0.0), vb=(v2, 0.0, 0.0))
    o = Oracle(p)
    fs, R = S.static_features(o)
    dx, dy = 1 / 6, 1 / 5
    Rw = 2 * d / dx ** 2 + 2 * d / dy ** 2 + abs(v1) / dx + abs(v2) / dy
    np.testing.assert_allclose(R, Rw, rtol=1e-14)
    want = [2 * d / dx ** 2 / Rw, 2 * d / dy ** 2 / Rw, v1 / dx / Rw, v2 / dy / Rw, d, 0, 0, 0, 0, o.tau() * Rw]
    np.testing.assert_allclose(fs, np.tile(want, (len(fs), 1)), rtol=1e-13, atol=1e-16)


def test_rate_closed_form_with_a_cross_term_and_reaction():
    """Identity map, constant tensor D = d [[1, c], [c, 1]], v constant, f0: the
    rate is R = 2d/dxi^2 + 2d/deta^2 + 2 c d/(dxi deta) + |v1|/dxi + |v2|/deta
    + |f0| (beta = 2 c d, phi = f0) and every one of its terms is positive."""
    d, c, v1, v2, f0 = 0.04, 0.3, -0.7, 1.2, -0.9
    p = W.base(n_xi=6, n_eta=5, M=(1.0, c, 1.0), d_aff=(d, 0.0, 0.0), va=(v1, 0.0, 0.0), vb=(v2, 0.0, 0.0),
               f0=f0)
    o = Oracle(p)
    fs, R = S.static_features(o)
    dx, dy = 1 / 6, 1 / 5
    Rw = 2 * d / dx ** 2 + 2 * d / dy ** 2 + 2 * c * d / (dx * dy) + abs(v1) / dx + abs(v2) / dy + abs(f0)
    np.testing.assert_allclose(R, Rw, rtol=1e-13)
    want = [2 * d / dx ** 2 / Rw, 2 * d / dy ** 2 / Rw, v1 / dx / Rw, v2 / dy / Rw]
    np.testing.assert_allclose(fs[:, :4], np.tile(want, (len(fs), 1)), rtol=1e-13)


def test_edge_samples_of_a_diffusivity_linear_in_x():
    """Identity map, D = (d0 + a x) I, v = 0, f = 0: half the trace at the
    centre is d0 + a x_c; its relative change is +-a (h_xi/2) / (d0 + a x_c)
    at the E and W edge midpoints and 0 at N and S; nu = -a enters R."""
    d0, a = 0.2, 0.15
    p = W.base(n_xi=6, n_eta=5, d_aff=(d0, a, 0.0), h_ratio_xi=0.3)
    o = Oracle(p)
    fs, R = S.static_features(o)
    I, J = o.patch_nodes()
    dx, dy = 1 / 6, 1 / 5
    xc = I * dx
    dc = d0 + a * xc
    rel = a * (0.3 * dx / 2) / dc
    np.testing.assert_allclose(fs[:, 4], dc, rtol=1e-13)
    np.testing.assert_allclose(fs[:, 5], rel, rtol=1e-12)
    np.testing.assert_allclose(fs[:, 6], -rel, rtol=1e-12)
    np.testing.assert_allclose(fs[:, 7:9], 0.0, atol=1e-14)
    np.testing.assert_allclose(R, 2 * dc / dx ** 2 + 2 * dc / dy ** 2 + a / dx, rtol=1e-13)
    np.testing.assert_allclose(fs[:, 9], o.tau() * R, rtol=1e-13)


def test_metric_features_multiply_the_matching_differences():
    p = W.c5_surrogate_field(n_r=6, n_theta=12, m=5)
    o = Oracle(p)
    U = o.init_field()
    fs, R = S.static_features(o)
    X, s, R2 = S.features(o, U)
    x, s2 = S.stencil_features(S.stencils(o, U))
    np.testing.assert_array_equal(R, R2)
    np.testing.assert_array_equal(s, s2)
    for col, k in ((25, 2), (26, 10), (27, 1), (28, 5)):
        np.testing.assert_array_equal(X[:, col], fs[:, col - 25] * x[:, k])
    np.testing.assert_array_equal(X[:, 29:], fs[:, 4:])


def test_features_of_a_patch_subset_are_the_rows_of_the_full_set():
    p = W.c5_surrogate_field(n_r=6, n_theta=12, m=5)
    o = Oracle(p)
    U = o.init_field()
    X, s, R = S.features(o, U)
    sel = np.array([0, 11, 12, 30, o.n_patch - 1])
    Xs, ss, Rs = S.features(o, U, sel=sel)
    np.testing.assert_array_equal(Xs, X[sel])
    np.testing.assert_array_equal(ss, s[sel])
    np.testing.assert_array_equal(Rs, R[sel])


def test_split_input_carries_sixteen_bits():
    x = np.random.default_rng(3).normal(size=(200, S.N_PAD)) * 10.0 ** np.random.default_rng(4).uniform(-3, 3, (200, S.N_PAD))
    hi, lo = S.split_input(x)
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.all(S.bf16(hi) == hi) and np.all(S.bf16(lo) == lo)
    assert np.all(np.abs(hi + lo - x32) <= 2.0 ** -16 * np.abs(x32))


def test_static_features_annulus_metric_terms_sum_to_one():
    """beta = phi = 0 on the annulus with v = 0, f = 0, so the four metric
    terms carry the whole rate R."""
    o = Oracle(W.c5_surrogate_field(n_r=7, n_theta=12, m=5))
    fs, R = S.static_features(o)
    np.testing.assert_allclose(np.abs(fs[:, :4]).sum(1), 1.0, rtol=1e-13)
    assert np.all(fs[:, 4] > 0.5)
    assert np.all(np.abs(fs[:, 5:9]) < 0.05)


def test_check_closed_form():
    F1 = np.array([1.0, -1.0, 0.0, 0.0])
    rho = math.sqrt(0.5)
    tol = 1e-3 * (np.abs(F1) + rho)
    inside = F1 + 0.999 * tol * np.array([1, -1, 1, -1])
    outside = F1 + 1.001 * tol * np.array([1, -1, 1, -1])
    assert S.check(inside, F1).all()
    assert not S.check(outside, F1).any()


def test_patch_F_is_independent_of_K_for_constant_diffusion():
    """Summation by parts: constant alpha, gamma and no other terms make the
    restricted F independent of the number of micro steps."""
    p = W.base(n_xi=7, n_eta=6, m_xi=7, m_eta=7, d_aff=(0.3, 0.0, 0.0), M=(1.0, 0.0, 2.0), init="bump")
    o = Oracle(p)
    U = o.init_field() + np.random.default_rng(1).normal(size=o.n_macro) * 0.01
    a = S.patch_F(o, U, 0.0)
    b = S.patch_F(o, U, 0.0, 1)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-11 * np.abs(a).max())


def _time_dependent_case():
    p = W.c2_heterogeneous(n=6, m=5, n_macro=3)
    p["src_amp"] = p["src_amp"] * 50.0           # a source that moves F within three steps
    return p


@pytest.mark.parametrize("case", ["annulus", "time_dependent_source"])
def test_all_fallback_surrogate_step_is_the_plain_scheme(case):
    p = W.c5_surrogate_field(n_r=6, n_theta=12, m=5) if case == "annulus" else _time_dependent_case()
    o = Oracle(p)
    U0 = o.init_field()
    dtm = o.dt_macro()
    th = _theta()
    mu, sig = np.zeros(S.N_IN), np.ones(S.N_IN)
    got, n_fb = S.surrogate_step(o, U0, 0.0, dtm, 3, th, mu, sig, 1.0, eps=-1.0)
    want = o.step(U0, 0.0, dtm, 3)
    assert n_fb == 3 * o.n_patch
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())
    if case != "annulus":
        return
    # with every patch accepted, F is the network's prediction scaled by R s
    X, s, R = S.features(o, U0)
    F, ok, F_hat, _ = S.surrogate_F(o, U0, 0.0, th, mu, sig, 2.0, eps=np.inf)
    assert ok.all()
    y, _ = S.forward(th, X)
    np.testing.assert_allclose(F, 2.0 * y * R * s, rtol=1e-15)


def test_network_input_is_standardised():
    """F-hat = y((x - mu) / sigma) y_scale R s with the standardisation applied
    before the network, for non-trivial mu and sigma."""
    p = W.c5_surrogate_field(n_r=6, n_theta=12, m=5)
    o = Oracle(p)
    U0 = o.init_field()
    th = _theta()
    rng = np.random.default_rng(5)
    mu, sig = rng.normal(size=S.N_IN) * 0.2, rng.uniform(0.5, 2.0, S.N_IN)
    X, s, R = S.features(o, U0)
    F, ok, F_hat, _ = S.surrogate_F(o, U0, 0.0, th, mu, sig, 1.5, eps=np.inf)
    y, _ = S.forward(th, (X - mu) / sig)
    np.testing.assert_allclose(F_hat, 1.5 * y * R * s, rtol=1e-14)
    y0, _ = S.forward(th, X)
    assert np.abs(F_hat - 1.5 * y0 * R * s).max() > 1e-6 * np.abs(F_hat).max()
