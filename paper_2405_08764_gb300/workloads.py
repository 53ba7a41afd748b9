"""Seeded synthetic workloads shaped like the paper's problems.

This module only holds parameter values and seeded random draws.  It contains
none of the patch-dynamics arithmetic: the CUDA library and the CPU oracle each
turn these plain dictionaries into their own descriptors and evaluate every
field themselves.

Problem dictionary keys (all plain Python values or numpy arrays):
  n_xi, n_eta, periodic_xi, box=(xi0, xi1, eta0, eta1)
  map in {"identity", "sine", "tanh", "polar"}, map_p (4 floats)
  m_xi, m_eta, h_ratio_xi, h_ratio_eta, k_micro, cfl_micro
  conv in {"upwind", "central"}, restrict in {"lifted", "macro"}
  M=(M11, M12, M22), d_aff=(d0, dx, dy), d_sin=(amp, k),
  four=dict(c=[...], phi=[...], ra=, rb=)   (up to 3 terms)
  va=(a0, a1, a2), vb=(b0, b1, b2), f0
  src in {"none", "mms_sinprod", "exp_linear", "gauss_patch"}, src_p (3), src_amp (array or None)
  time in {"const", "exp", "sin"}, tc
  sol in {"none", "exp_xyt", "sinprod_decay"}
  init in {"zero", "exact", "bessel", "bump", "annulus_poly"}, init_p (list of floats)
  micro in {"fe", "adi"} (micro time stepper), dt_micro (float or None = cfl rule)
  q_refresh (edge data refreshed q times per burst, 1 = fixed)
  dt_macro (float or None = suggested), n_macro, t0
"""
from __future__ import annotations

import math

import numpy as np

MAPS = {"identity": 0, "sine": 1, "tanh": 2, "polar": 3}
CONV = {"upwind": 0, "central": 1}
RESTRICT = {"lifted": 0, "macro": 1}
SRC = {"none": 0, "mms_sinprod": 1, "exp_linear": 2, "gauss_patch": 3}
TIME = {"const": 0, "exp": 1, "sin": 2}
SOL = {"none": 0, "exp_xyt": 1, "sinprod_decay": 2}
INIT = {"zero": 0, "exact": 1, "bessel": 2, "bump": 3, "annulus_poly": 4}


def base(**kw) -> dict:
    p = dict(
        n_xi=8, n_eta=8, periodic_xi=0, box=(0.0, 1.0, 0.0, 1.0),
        map="identity", map_p=(0.0, 0.0, 0.0, 0.0),
        m_xi=7, m_eta=7, h_ratio_xi=0.2, h_ratio_eta=0.2, k_micro=20, cfl_micro=0.4,
        conv="upwind", restrict="lifted",
        M=(1.0, 0.0, 1.0), d_aff=(1.0, 0.0, 0.0), d_sin=(0.0, 1.0),
        four=dict(c=[], phi=[], ra=1.0, rb=2.0),
        va=(0.0, 0.0, 0.0), vb=(0.0, 0.0, 0.0), f0=0.0,
        src="none", src_p=(0.0, 0.0, 0.0), src_amp=None,
        time="const", tc=0.0, sol="none", init="zero", init_p=[],
        micro="fe", dt_micro=None, q_refresh=1,
        dt_macro=None, n_macro=1, t0=0.0,
    )
    p.update(kw)
    return p


def n_patch(p: dict) -> int:
    cols = p["n_xi"] if p["periodic_xi"] else p["n_xi"] - 1
    return cols * (p["n_eta"] - 1)


def n_macro_nodes(p: dict) -> int:
    nx = p["n_xi"] if p["periodic_xi"] else p["n_xi"] + 1
    return nx * (p["n_eta"] + 1)


# --------------------------------------------------------------------------
# the five workloads


def c1_manufactured(n: int = 8, m: int = 7, n_macro: int = 50, dt_macro: float = 0.01) -> dict:
    """Plain patch scheme on [0,1]^2, identity map, D = 0.05 I, v = (1,1), f = 0,
    manufactured u = exp(-t) sin(pi x) sin(pi y), Dirichlet data, 50 steps to t = 0.5."""
    return base(
        n_xi=n, n_eta=n, m_xi=m, m_eta=m, h_ratio_xi=0.2, h_ratio_eta=0.2,
        M=(1.0, 0.0, 1.0), d_aff=(0.05, 0.0, 0.0), va=(1.0, 0.0, 0.0), vb=(1.0, 0.0, 0.0),
        src="mms_sinprod", time="exp", tc=-1.0, sol="sinprod_decay", init="exact",
        dt_macro=dt_macro, n_macro=n_macro,
    )


def c2_heterogeneous(n: int = 64, m: int = 11, n_macro: int = 200, seed: int = 2) -> dict:
    """Convection-dominated heterogeneous CDR on [0,1]^2 with a tanh stretching
    (factor 3) clustered at x = 1 and y = 1; tensor diffusion
    1e-3 (1 + 0.5 sin 2pi x sin 2pi y) [[1, .2], [.2, 1]], v = (1 + x/2, 1 + y/2),
    source sin(pi t) exp(-(x^2 + y^2)) times a seeded U[0.5, 1.5] amplitude per
    patch, u = 0 on the boundary and at t = 0."""
    p = base(
        n_xi=n, n_eta=n, map="tanh", map_p=(3.0, 3.0, 0.0, 0.0), m_xi=m, m_eta=m,
        M=(1.0, 0.2, 1.0), d_aff=(1e-3, 0.0, 0.0), d_sin=(0.5e-3, 1.0),
        va=(1.0, 0.5, 0.0), vb=(1.0, 0.0, 0.5), f0=0.0,
        src="gauss_patch", time="sin", tc=math.pi, sol="none", init="zero",
        n_macro=n_macro,
    )
    rng = np.random.default_rng(seed)
    p["src_amp"] = rng.uniform(0.5, 1.5, n_patch(p))
    return p


def c3_annulus(n_r: int = 127, n_theta: int = 512, m: int = 9, seed: int = 3,
               t_final: float = 0.02, n_modes: int = 4) -> dict:
    """Non-axisymmetric diffusion in the annulus 1 <= r <= 2 (polar map,
    xi = theta periodic, eta in [0,1] with a radial tanh stretch 1.5), initial
    data sum_k a_k Z_k(mu_k r) cos(k theta), seeded a_k ~ U[0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    amps = rng.uniform(0.5, 1.5, n_modes)
    return base(
        n_xi=n_theta, n_eta=n_r, periodic_xi=1, box=(0.0, 2.0 * math.pi, 0.0, 1.0),
        map="polar", map_p=(1.0, 2.0, 1.5, 0.0), m_xi=m, m_eta=m,
        M=(1.0, 0.0, 1.0), d_aff=(1.0, 0.0, 0.0), conv="central",
        init="bessel", init_p=[float(n_modes), 1.0, 2.0] + [float(a) for a in amps],
        t_final=t_final,
    )


def c4_instance(inst: int, seed0: int = 4) -> dict:
    """One of the 4096 uneven batched instances (seed 4 + instance id)."""
    rng = np.random.default_rng(seed0 + inst)
    n = int(rng.choice([16, 32, 64, 128]))
    kind = int(rng.integers(0, 3))
    m = int(rng.choice([5, 7, 9, 11]))
    lam = 10.0 ** rng.uniform(-4.0, -1.0, 2)
    th = rng.uniform(0.0, math.pi)
    c, s = math.cos(th), math.sin(th)
    M = (lam[0] * c * c + lam[1] * s * s, (lam[0] - lam[1]) * c * s, lam[0] * s * s + lam[1] * c * c)
    v = rng.uniform(-2.0, 2.0, 2)
    f = float(rng.uniform(0.0, 1.0))
    p = base(
        n_xi=n, n_eta=n, m_xi=m, m_eta=m, M=M, d_aff=(1.0, 0.0, 0.0),
        va=(float(v[0]), 0.0, 0.0), vb=(float(v[1]), 0.0, 0.0), f0=f,
        init="bump", n_macro=100,
    )
    if kind == 1:
        st = float(rng.uniform(1.0, 4.0))
        p.update(map="tanh", map_p=(st, st, 0.0, 0.0))
    elif kind == 2:
        ra = float(rng.uniform(0.5, 1.0))
        rb = float(rng.uniform(1.5, 3.0))
        p.update(map="polar", map_p=(ra, rb, 0.0, 0.0), periodic_xi=1,
                 box=(0.0, 2.0 * math.pi, 0.0, 1.0))
    return p


def c4_batch(n_inst: int = 4096, seed0: int = 4) -> list:
    return [c4_instance(i, seed0) for i in range(n_inst)]


def c5_surrogate_field(n_r: int = 511, n_theta: int = 2048, m: int = 9, seed: int = 5,
                       n_macro: int = 100) -> dict:
    """Annulus 512 radial x 2048 angular nodes with a seeded smooth diffusivity
    D(r, theta) = 1 + sum_{k<=3} c_k cos(k theta + phi_k) cos(k pi rho(r))."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.1, 0.1, 3)
    ph = rng.uniform(0.0, 2.0 * math.pi, 3)
    amps = rng.uniform(0.5, 1.5, 4)
    return base(
        n_xi=n_theta, n_eta=n_r, periodic_xi=1, box=(0.0, 2.0 * math.pi, 0.0, 1.0),
        map="polar", map_p=(1.0, 2.0, 1.5, 0.0), m_xi=m, m_eta=m,
        M=(1.0, 0.0, 1.0), d_aff=(1.0, 0.0, 0.0),
        four=dict(c=[float(x) for x in c], phi=[float(x) for x in ph], ra=1.0, rb=2.0),
        conv="central", init="bessel", init_p=[4.0, 1.0, 2.0] + [float(a) for a in amps],
        n_macro=n_macro,
    )


# --------------------------------------------------------------------------
# the paper's own test problems (Section 4)


def paper_cdr(variable_d: bool, lam: float = 0.1, n: int = 10, m: int = 11,
              h_ratio: float = 0.01, k_micro: int = 20, cfl: float = 0.4) -> dict:
    """Section 4.1: D = 1 (4.1.1) or D = 1 + x (4.1.2), v = (10x, 10y) or
    (1 + 10x, 10y), f = 20, exact solution exp(x + y + t), sine stretching lambda."""
    if variable_d:
        d_aff, va, src_p = (1.0, 1.0, 0.0), (1.0, 10.0, 0.0), (-1.0, 8.0, 10.0)
    else:
        d_aff, va, src_p = (1.0, 0.0, 0.0), (0.0, 10.0, 0.0), (-1.0, 10.0, 10.0)
    return base(
        n_xi=n, n_eta=n, map="sine", map_p=(lam, 0.0, 0.0, 0.0), m_xi=m, m_eta=m,
        h_ratio_xi=h_ratio, h_ratio_eta=h_ratio, k_micro=k_micro, cfl_micro=cfl,
        d_aff=d_aff, va=va, vb=(0.0, 0.0, 10.0), f0=20.0,
        src="exp_linear", src_p=src_p, time="exp", tc=1.0, sol="exp_xyt", init="exact",
    )


def paper_cdr_adi(variable_d: bool, lam: float, n: int, n_t: int, restrict: str = "macro") -> dict:
    """Section 4.1 at the paper's own patch settings: h = 1e-3 in the
    computational box, n = 10 nano intervals, bursts of tau = 1e-6 made of
    n_t = 2 ADI nano steps, N_t macro steps of 1 / N_t over [0, 1]; the
    restriction reference is the macro value (eq. Time_Derivative as printed)."""
    p = paper_cdr(variable_d, lam=lam, n=n, m=11, h_ratio=1e-3 * n, k_micro=2)
    p.update(micro="adi", dt_micro=5e-7, restrict=restrict, dt_macro=1.0 / n_t, n_macro=n_t)
    return p


def paper_annulus(n_theta: int = 16, n_r: int = 10, m: int = 9, h_ratio: float = 0.2) -> dict:
    """Section 4.2: diffusion in 1 <= r <= 2 with x = eta cos xi, y = eta sin xi,
    initial data (r - 1)(2 - r) sin(theta), zero data on both circles."""
    return base(
        n_xi=n_theta, n_eta=n_r, periodic_xi=1, box=(0.0, 2.0 * math.pi, 1.0, 2.0),
        map="polar", map_p=(1.0, 2.0, 0.0, 0.0), m_xi=m, m_eta=m,
        h_ratio_xi=h_ratio, h_ratio_eta=h_ratio, conv="central",
        init="annulus_poly", init_p=[1.0, 2.0],
    )


def bench_workload() -> dict:
    """The single-GPU benchmark workload: the 65 x 65 tanh-stretched
    heterogeneous tensor-diffusion problem, 11 x 11 micro points, 200 steps."""
    return c2_heterogeneous()
