"""Pins of the edge-data refresh (Q > 1) of the oracle.

For constant alpha, gamma and no convection, reaction or source, with the
lifted restriction reference, summation by parts makes each micro step change
the trapezoid average of a patch by dt times a 9-point macro stencil S applied
to the field whose interpolant supplied the edge data.  With the edge data
rebuilt Q times per burst from V_q = U + (restricted change so far), Dirichlet
data at the sub-burst start times, the restricted change of a burst is
therefore exactly Q forward-Euler sub-steps of size tau / Q of dV/dt = S(V);
a source s(t) G adds dt s(t_k) times the patch's trapezoid average of G per
micro step.  Also: the split form equals the literal form, Q = 1 is the
fixed-edge scheme, and the refresh changes F by an amount that shrinks
linearly with tau."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W


def _sbp_problem(periodic, Q, source, K=12):
    box = (0.0, 2.0 * math.pi, 0.0, 1.0) if periodic else (0.0, 1.0, 0.0, 1.0)
    src = dict(src="exp_linear", src_p=(1.0, 0.5, -0.5), time="exp", tc=4.0) if source else {}
    return W.base(n_xi=7, n_eta=6, periodic_xi=periodic, box=box, m_xi=7, m_eta=5, h_ratio_xi=0.35,
                  h_ratio_eta=0.25, k_micro=K, M=(0.8, 0.0, 1.7), d_aff=(1.0, 0.0, 0.0),
                  sol="none" if periodic else "exp_xyt", init="zero", q_refresh=Q, **src)


def _trapezoid_G(o):
    """trapezoid average of the source factor G over every patch"""
    xi, eta = o.micro_coords()
    G = np.array([o.coeffs(a, b)[6] for a, b in zip(xi, eta)]).reshape(o.n_patch, o.my, o.mx)
    wa = np.ones(o.mx)
    wa[[0, -1]] = 0.5
    wb = np.ones(o.my)
    wb[[0, -1]] = 0.5
    return np.einsum("pba,b,a->p", G, wb, wa) / ((o.mx - 1) * (o.my - 1))


def _stencil_S(p, o, V):
    """the 9-point macro operator of the summation-by-parts closed form"""
    Dx = (p["box"][1] - p["box"][0]) / p["n_xi"]
    Dy = (p["box"][3] - p["box"][2]) / p["n_eta"]
    hx, hy = p["h_ratio_xi"] * Dx, p["h_ratio_eta"] * Dy
    dx, dy = hx / (p["m_xi"] - 1), hy / (p["m_eta"] - 1)
    wx1 = (hx ** 2 / 12 + dx ** 2 / 6) / (2 * Dx ** 2)
    wy1 = (hy ** 2 / 12 + dy ** 2 / 6) / (2 * Dy ** 2)
    wx = {-1: wx1, 0: 1 - 2 * wx1, 1: wx1}
    wy = {-1: wy1, 0: 1 - 2 * wy1, 1: wy1}
    Vg = V.reshape(o.nyp, o.nxp)
    I, J = o.patch_nodes()
    out = np.zeros(o.n_patch)
    for k, (i, j) in enumerate(zip(I, J)):
        def v(ii, jj):
            return Vg[jj, ii % o.nxp] if p["periodic_xi"] else Vg[jj, ii]
        sx = sum(wy[q] * (v(i + 1, j + q) - 2 * v(i, j + q) + v(i - 1, j + q)) for q in (-1, 0, 1))
        sy = sum(wx[q] * (v(i + q, j + 1) - 2 * v(i + q, j) + v(i + q, j - 1)) for q in (-1, 0, 1))
        out[k] = p["M"][0] * sx / Dx ** 2 + p["M"][2] * sy / Dy ** 2
    return out


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 12])
@pytest.mark.parametrize("periodic,source", [(0, False), (1, False), (0, True)])
def test_refresh_is_macro_substepping_under_summation_by_parts(orc, Q, periodic, source):
    """with a source s(t) G each micro step adds dt s(t_k) times the trapezoid
    average of G, which also pins the time levels of the sub-bursts"""
    p = _sbp_problem(periodic, Q, source)
    o = orc.Oracle(p)
    trG = _trapezoid_G(o) if source else None
    rng = np.random.default_rng(7)
    T = 0.3
    U = o.apply_bc(rng.normal(size=o.n_macro), T)
    dt = 0.8 * o.dt_micro()
    K = p["k_micro"]
    tau, Ks = K * dt, K // Q
    dtm = 2.5e-4
    got = o.step(U, T, dtm, 1, dt_micro=dt)
    # Q forward-Euler sub-steps of the macro stencil, boundary data at the sub-times
    I, J = o.patch_nodes()
    nodes = J * o.nxp + I
    dR = np.zeros(o.n_patch)
    for q in range(Q):
        V = U.copy()
        if q > 0:
            V[nodes] += dR
            V = o.apply_bc(V, T + q * Ks * dt)
        dR = dR + Ks * dt * _stencil_S(p, o, V)
        if source:
            for k in range(Ks):
                dR = dR + dt * o.time_factor(T + (q * Ks + k) * dt) * trG
    want = U.copy()
    want[nodes] += dtm * dR / tau
    want = o.apply_bc(want, T + dtm)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def _tensor_problem(Q, restrict="lifted"):
    p = W.c2_heterogeneous(n=8, m=7, n_macro=2)
    p.update(k_micro=12, q_refresh=Q, restrict=restrict, sol="exp_xyt")
    return p


@pytest.mark.parametrize("Q", [2, 3, 12])
@pytest.mark.parametrize("restrict", ["lifted", "macro"])
def test_refresh_split_form_equals_literal_form(orc, Q, restrict):
    p = _tensor_problem(Q, restrict)
    o = orc.Oracle(p)
    U = o.apply_bc(o.init_field() + 0.3 * np.random.default_rng(1).normal(size=o.n_macro), 0.1)
    dtm = 0.5 * o.dt_macro()
    a = o.step(U, 0.1, dtm, 2, form="split")
    b = o.step(U, 0.1, dtm, 2, form="literal")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_refresh_changes_the_step_and_the_change_shrinks_with_tau(orc):
    """Q = 1 through the refresh code equals the fixed-edge scheme; the Q = 3
    step differs from it by O(tau) in F (the edge data move by O(tau))."""
    diffs = []
    for cfl in (0.4, 0.2, 0.1):
        base = dict(_tensor_problem(1), cfl_micro=cfl)
        o1 = orc.Oracle(base)
        o3 = orc.Oracle(dict(base, q_refresh=3))
        U = o1.apply_bc(o1.init_field() + 0.3 * np.random.default_rng(2).normal(size=o1.n_macro), 0.0)
        dtm = 0.5 * o1.dt_macro()
        a, b = o1.step(U, 0.0, dtm, 1), o3.step(U, 0.0, dtm, 1)
        F1, F3 = (a - U) / dtm, (b - U) / dtm
        diffs.append(np.linalg.norm(F3 - F1) / np.linalg.norm(F1))
    assert diffs[0] > 1e-6, diffs
    r = [diffs[k] / diffs[k + 1] for k in range(2)]
    assert all(1.7 < q < 2.3 for q in r), (diffs, r)


def test_refresh_descriptor_checks(orc):
    p = _tensor_problem(5)                        # 12 steps are not divisible by 5
    with pytest.raises(ValueError):
        orc.Oracle(p)
    with pytest.raises(ValueError):
        orc.Oracle(dict(_tensor_problem(3), micro="adi"))


@pytest.mark.parametrize("Q", [2, 4])
def test_refresh_macro_reference_adds_the_lift_bias(orc, Q):
    """Reading G4 with Q > 1: the sub-bursts are the same in both restriction
    modes, so one refreshed macro step with the paper-literal reference
    U^0 = U_ij differs from the lifted one at every interior node by
    dt_macro / tau times the bias (dxi^2 U_xixi + deta^2 U_etaeta) / 12 of the
    step's starting field, and not at all on the boundary."""
    pl, pm = _tensor_problem(Q), _tensor_problem(Q, "macro")
    ol, om = orc.Oracle(pl), orc.Oracle(pm)
    U = ol.apply_bc(ol.init_field() + 0.3 * np.random.default_rng(2).normal(size=ol.n_macro), 0.1)
    dtm = 0.5 * ol.dt_macro()
    diff = (om.step(U, 0.1, dtm, 1) - ol.step(U, 0.1, dtm, 1)).reshape(ol.nyp, ol.nxp)
    Ug = U.reshape(ol.nyp, ol.nxp)
    Dx, Dy = 1.0 / pl["n_xi"], 1.0 / pl["n_eta"]
    dx, dy = pl["h_ratio_xi"] * Dx / (pl["m_xi"] - 1), pl["h_ratio_eta"] * Dy / (pl["m_eta"] - 1)
    uxx = (Ug[1:-1, 2:] - 2 * Ug[1:-1, 1:-1] + Ug[1:-1, :-2]) / Dx ** 2
    uyy = (Ug[2:, 1:-1] - 2 * Ug[1:-1, 1:-1] + Ug[:-2, 1:-1]) / Dy ** 2
    want = dtm / ol.tau() * (dx * dx * uxx + dy * dy * uyy) / 12.0
    np.testing.assert_allclose(diff[1:-1, 1:-1], want, rtol=1e-8, atol=1e-12 * np.abs(want).max())
    inner = np.zeros_like(diff, dtype=bool)
    inner[1:-1, 1:-1] = True
    assert np.all(diff[~inner] == 0.0)
