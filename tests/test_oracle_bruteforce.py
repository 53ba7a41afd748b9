"""Brute force on tiny grids: the whole macro step of Section 3 rebuilt as dense
matrices with numpy (interpolant by a 9x9 Vandermonde solve, ghost points as
affine maps of the patch interior, forward Euler as repeated matrix products,
trapezoid rule as a weight vector) and compared with the oracle's loop code.
Covers the cross term and the ghost corners (beta != 0), both upwind
directions, reaction, a time-dependent source, Dirichlet data, periodic wrap
and both restriction references."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W


def _time_factor(p, t):
    if p["time"] == "exp":
        return math.exp(p["tc"] * t)
    if p["time"] == "sin":
        return math.sin(p["tc"] * t)
    return 1.0


def dense_step(o, p, U, T, dtm, dt):
    s = o.s
    mx, my = s.m_xi, s.m_eta
    nx, ny = mx - 1, my - 1
    Dx = (s.xi1 - s.xi0) / s.n_xi
    Dy = (s.eta1 - s.eta0) / s.n_eta
    hx, hy = s.h_ratio_xi * Dx, s.h_ratio_eta * Dy
    dx, dy = hx / nx, hy / ny
    K = s.k_micro
    nxp = o.nxp
    Ug = U.reshape(o.nyp, nxp)
    # monomial basis s^k t^l, (k, l) in 0..2
    kl = [(k, l) for k in range(3) for l in range(3)]
    V = np.array([[(pp * Dx) ** k * (q * Dy) ** l for (k, l) in kl]
                  for pp in (-1, 0, 1) for q in (-1, 0, 1)])
    Vinv = np.linalg.inv(V)
    n_int = mx * my

    def idx(a, b):
        return b * mx + a

    ii, jj = o.patch_nodes()
    Unew = U.copy()
    wx = np.ones(mx); wx[[0, -1]] = 0.5
    wy = np.ones(my); wy[[0, -1]] = 0.5
    wtrap = (wy[:, None] * wx[None, :]).ravel() / (nx * ny)
    for pch in range(o.n_patch):
        i, j = ii[pch], jj[pch]
        vals = np.array([Ug[j + q, (i + pp) % nxp] for pp in (-1, 0, 1) for q in (-1, 0, 1)])
        c = dict(zip(kl, Vinv @ vals))

        def dPs(sv, tv):
            return sum(c[(k, l)] * k * sv ** (k - 1) * tv ** l for (k, l) in kl if k > 0)

        def dPt(sv, tv):
            return sum(c[(k, l)] * l * sv ** k * tv ** (l - 1) for (k, l) in kl if l > 0)

        sa = [-0.5 * hx + a * dx for a in range(-1, mx + 1)]
        tb = [-0.5 * hy + b * dy for b in range(-1, my + 1)]
        # lift from the Taylor coefficients of the interpolant at the centre
        Ux, Uy, Uxx, Uyy, Uxy = c[(1, 0)], c[(0, 1)], 2 * c[(2, 0)], 2 * c[(0, 2)], c[(1, 1)]
        C0 = c[(0, 0)] - hx * hx * Uxx / 24 - hy * hy * Uyy / 24
        u0 = np.array([C0 + sa[a + 1] * Ux + tb[b + 1] * Uy
                       + 0.5 * (sa[a + 1] ** 2 * Uxx + 2 * sa[a + 1] * tb[b + 1] * Uxy + tb[b + 1] ** 2 * Uyy)
                       for b in range(my) for a in range(mx)])
        # extended-grid values as affine maps (row, const) of the interior
        ext = {}
        for b in range(my):
            for a in range(mx):
                e = np.zeros(n_int); e[idx(a, b)] = 1.0
                ext[(a, b)] = (e, 0.0)
        for a in range(mx):
            r, k0 = ext[(a, 1)]
            ext[(a, -1)] = (r, k0 - 2 * dy * dPt(sa[a + 1], -hy / 2))
            r, k0 = ext[(a, ny - 1)]
            ext[(a, ny + 1)] = (r, k0 + 2 * dy * dPt(sa[a + 1], hy / 2))
        for b in range(-1, my + 1):
            r, k0 = ext[(1, b)]
            ext[(-1, b)] = (r, k0 - 2 * dx * dPs(-hx / 2, tb[b + 1]))
            r, k0 = ext[(nx - 1, b)]
            ext[(nx + 1, b)] = (r, k0 + 2 * dx * dPs(hx / 2, tb[b + 1]))
        # operator rows
        Lm = np.zeros((n_int, n_int))
        lv = np.zeros(n_int)
        G = np.zeros(n_int)
        amp = p["src_amp"][pch] if p.get("src_amp") is not None else 1.0
        for b in range(my):
            for a in range(mx):
                co = o.coeffs(s.xi0 + i * Dx - 0.5 * hx + a * dx, s.eta0 + j * Dy - 0.5 * hy + b * dy)
                al, be, ga, nu, om, ph, g = co
                wts = {(0, 0): -2 * al / dx ** 2 - 2 * ga / dy ** 2 + ph,
                       (1, 0): al / dx ** 2, (-1, 0): al / dx ** 2,
                       (0, 1): ga / dy ** 2, (0, -1): ga / dy ** 2,
                       (1, 1): be / (4 * dx * dy), (-1, -1): be / (4 * dx * dy),
                       (1, -1): -be / (4 * dx * dy), (-1, 1): -be / (4 * dx * dy)}
                if p["conv"] == "central":
                    wts[(1, 0)] -= nu / (2 * dx); wts[(-1, 0)] += nu / (2 * dx)
                    wts[(0, 1)] -= om / (2 * dy); wts[(0, -1)] += om / (2 * dy)
                else:
                    if nu > 0:
                        wts[(0, 0)] -= nu / dx; wts[(-1, 0)] += nu / dx
                    else:
                        wts[(0, 0)] += nu / dx; wts[(1, 0)] -= nu / dx
                    if om > 0:
                        wts[(0, 0)] -= om / dy; wts[(0, -1)] += om / dy
                    else:
                        wts[(0, 0)] += om / dy; wts[(0, 1)] -= om / dy
                for (da, db), wv in wts.items():
                    r, k0 = ext[(a + da, b + db)]
                    Lm[idx(a, b)] += wv * r
                    lv[idx(a, b)] += wv * k0
                G[idx(a, b)] = amp * g
        u = u0.copy()
        for k in range(K):
            u = u + dt * (Lm @ u + lv + _time_factor(p, T + k * dt) * G)
        ref = wtrap @ u0 if p["restrict"] == "lifted" else Ug[j, i]
        dU = wtrap @ u - ref
        Unew[j * nxp + i] = U[j * nxp + i] + dtm * dU / (K * dt)
    return o.apply_bc(Unew, T + dtm)


CASES = {
    "tanh_tensor_mms": W.base(
        n_xi=4, n_eta=4, m_xi=3, m_eta=4, k_micro=2, h_ratio_xi=0.4, h_ratio_eta=0.3,
        map="tanh", map_p=(2.0, 1.2, 0, 0), M=(1.0, 0.35, 0.7), d_aff=(0.3, 0.2, -0.1),
        d_sin=(0.05, 1.0), va=(0.4, 1.0, -0.6), vb=(-0.3, 0.5, 0.4), f0=0.6,
        src="mms_sinprod", time="exp", tc=-1.0, sol="sinprod_decay"),
    "macro_restrict": W.base(
        n_xi=4, n_eta=5, m_xi=5, m_eta=3, k_micro=3, restrict="macro",
        M=(0.5, -0.2, 1.0), va=(-1.0, 0.3, 0.0), vb=(0.7, 0.0, -0.4), f0=-0.3,
        src="exp_linear", src_p=(-1.0, 8.0, 10.0), time="exp", tc=1.0, sol="exp_xyt",
        map="sine", map_p=(0.3, 0, 0, 0)),
    "polar_periodic_gauss": W.base(
        n_xi=5, n_eta=4, periodic_xi=1, box=(0.0, 2 * math.pi, 0.0, 1.0), map="polar",
        map_p=(0.8, 1.9, 1.2, 0), m_xi=4, m_eta=3, k_micro=2, conv="central",
        M=(1.0, 0.25, 0.6), four=dict(c=[0.1, -0.05, 0.02], phi=[0.1, 0.5, 0.9], ra=0.8, rb=1.9),
        va=(0.2, 0.3, 0.0), vb=(0.0, 0.0, 0.1), src="gauss_patch", time="sin", tc=math.pi),
}


@pytest.mark.parametrize("name", list(CASES))
def test_oracle_step_equals_dense_matrix_formulation(orc, name):
    p = dict(CASES[name])
    if p["src"] == "gauss_patch":
        p["src_amp"] = np.random.default_rng(7).uniform(0.5, 1.5, W.n_patch(p))
    o = orc.Oracle(p)
    rng = np.random.default_rng(3)
    U = o.apply_bc(1.0 + 0.3 * rng.normal(size=o.n_macro), 0.25)
    dt, dtm = o.dt_micro(), 0.5 * o.dt_macro()
    want = dense_step(o, p, U, 0.25, dtm, dt)
    got = o.step(U, 0.25, dtm, 1, dt, form="literal")
    got_split = o.step(U, 0.25, dtm, 1, dt, form="split")
    scale = np.abs(want).max()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(got_split, want, rtol=0, atol=1e-12 * scale)
