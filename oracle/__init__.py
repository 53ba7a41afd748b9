"""Python access to the plain FP64 CPU oracle (oracle/pd_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the product library never imports it.  The C source
is compiled with gcc (no CUDA, no shared headers with the GPU library).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libpd_oracle.so")
_lock = threading.Lock()
_lib = None

MAPS = {"identity": 0, "sine": 1, "tanh": 2, "polar": 3}
CONV = {"upwind": 0, "central": 1}
RESTRICT = {"lifted": 0, "macro": 1}
SRC = {"none": 0, "mms_sinprod": 1, "exp_linear": 2, "gauss_patch": 3}
TIME = {"const": 0, "exp": 1, "sin": 2}
SOL = {"none": 0, "exp_xyt": 1, "sinprod_decay": 2}
INIT = {"zero": 0, "exact": 1, "bessel": 2, "bump": 3, "annulus_poly": 4}
FORM = {"split": 0, "literal": 1}
MICRO = {"fe": 0, "adi": 1}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libpd_oracle.so."""
    src = os.path.join(_HERE, "pd_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "pd_oracle.h"))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Problem(C.Structure):
    _fields_ = [
        ("n_xi", C.c_int), ("n_eta", C.c_int), ("periodic_xi", C.c_int),
        ("xi0", C.c_double), ("xi1", C.c_double), ("eta0", C.c_double), ("eta1", C.c_double),
        ("map", C.c_int), ("map_p", C.c_double * 4),
        ("m_xi", C.c_int), ("m_eta", C.c_int),
        ("h_ratio_xi", C.c_double), ("h_ratio_eta", C.c_double),
        ("k_micro", C.c_int), ("cfl_micro", C.c_double),
        ("conv", C.c_int), ("restrict_mode", C.c_int),
        ("M11", C.c_double), ("M12", C.c_double), ("M22", C.c_double),
        ("d0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("ds", C.c_double), ("dk", C.c_double),
        ("n_four", C.c_int), ("four_c", C.c_double * 3), ("four_phi", C.c_double * 3),
        ("four_ra", C.c_double), ("four_rb", C.c_double),
        ("va", C.c_double * 3), ("vb", C.c_double * 3), ("f0", C.c_double),
        ("src", C.c_int), ("src_p", C.c_double * 3), ("src_amp", C.POINTER(C.c_double)),
        ("tkind", C.c_int), ("tc", C.c_double),
        ("sol", C.c_int),
        ("micro", C.c_int), ("dt_micro_fixed", C.c_double),
        ("q_refresh", C.c_int),
    ]


_D = C.POINTER(C.c_double)
_P = C.POINTER(Problem)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ORC_SO_OVERRIDE") or build()
            L = C.CDLL(path)
            sig = {
                "orc_n_patch": (C.c_int, [_P]), "orc_n_macro": (C.c_int, [_P]),
                "orc_validate": (C.c_int, [_P]),
                "orc_map": (None, [_P, C.c_double, C.c_double, _D]),
                "orc_coeffs": (None, [_P, C.c_double, C.c_double, _D]),
                "orc_physical": (None, [_P, C.c_double, C.c_double, _D]),
                "orc_time_factor": (C.c_double, [_P, C.c_double]),
                "orc_exact": (C.c_double, [_P, C.c_double, C.c_double, C.c_double]),
                "orc_dt_micro": (C.c_double, [_P]), "orc_dt_macro": (C.c_double, [_P]),
                "orc_init_field": (None, [_P, C.c_int, _D, C.c_double, _D]),
                "orc_micro_coords": (None, [_P, _D, _D]),
                "orc_lift": (None, [_P, _D, _D, _D]),
                "orc_forcing": (None, [_P, _D, C.c_double, _D]),
                "orc_burst": (None, [_P, _D, C.c_double, C.c_int, C.c_double, C.c_int, _D]),
                "orc_restrict": (None, [_P, _D, _D, C.c_int, _D]),
                "orc_project": (None, [_P, _D, _D, C.c_double, C.c_double, C.c_double]),
                "orc_apply_bc": (None, [_P, _D, C.c_double]),
                "orc_step": (None, [_P, _D, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int]),
                "orc_full_domain_size": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "orc_full_domain": (None, [_P, C.c_int, _D, C.c_double, C.c_double, C.c_int]),
                "orc_micro_patch": (None, [_P, C.c_int, _D, _D, C.c_double, C.c_int, C.c_double, _D]),
                "orc_patch_dU": (None, [_P, _D, C.c_double, C.c_double, C.c_int, C.c_int,
                                        C.POINTER(C.c_int), _D]),
                "orc_bessel_root": (C.c_double, [C.c_int, C.c_double, C.c_double, C.c_int]),
                "orc_bessel_Z": (C.c_double, [C.c_int, C.c_double, C.c_double, C.c_double]),
                "orc_bessel_norm": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_int]),
                "orc_annulus_series": (C.c_double, [C.c_double, C.c_double, C.c_double,
                                                    C.c_double, C.c_double, C.c_int]),
                "orc_num_threads": (C.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


class Oracle:
    """One problem instance (a workloads dictionary) on the CPU oracle."""

    def __init__(self, prob: dict):
        self.prob = dict(prob)
        L = lib()
        s = Problem()
        p = self.prob
        s.n_xi, s.n_eta, s.periodic_xi = int(p["n_xi"]), int(p["n_eta"]), int(p["periodic_xi"])
        s.xi0, s.xi1, s.eta0, s.eta1 = [float(v) for v in p["box"]]
        s.map = MAPS[p["map"]]
        for k in range(4):
            s.map_p[k] = float(p["map_p"][k])
        s.m_xi, s.m_eta = int(p["m_xi"]), int(p["m_eta"])
        s.h_ratio_xi, s.h_ratio_eta = float(p["h_ratio_xi"]), float(p["h_ratio_eta"])
        s.k_micro, s.cfl_micro = int(p["k_micro"]), float(p["cfl_micro"])
        s.conv, s.restrict_mode = CONV[p["conv"]], RESTRICT[p["restrict"]]
        s.M11, s.M12, s.M22 = [float(v) for v in p["M"]]
        s.d0, s.dx, s.dy = [float(v) for v in p["d_aff"]]
        s.ds, s.dk = [float(v) for v in p["d_sin"]]
        four = p["four"]
        s.n_four = len(four["c"])
        for k in range(s.n_four):
            s.four_c[k] = float(four["c"][k])
            s.four_phi[k] = float(four["phi"][k])
        s.four_ra, s.four_rb = float(four["ra"]), float(four["rb"])
        for k in range(3):
            s.va[k] = float(p["va"][k])
            s.vb[k] = float(p["vb"][k])
            s.src_p[k] = float(p["src_p"][k])
        s.f0 = float(p["f0"])
        s.src = SRC[p["src"]]
        self._amp = None
        if p.get("src_amp") is not None:
            self._amp = np.ascontiguousarray(p["src_amp"], dtype=np.float64)
            s.src_amp = _dp(self._amp)
        s.tkind, s.tc = TIME[p["time"]], float(p["tc"])
        s.sol = SOL[p["sol"]]
        s.micro = MICRO[p.get("micro", "fe")]
        s.dt_micro_fixed = float(p.get("dt_micro") or 0.0)
        s.q_refresh = int(p.get("q_refresh") or 1)
        self.s = s
        self.L = L
        self._dt_micro = None
        rc = L.orc_validate(C.byref(s))
        if rc != 0:
            raise ValueError("invalid problem (code %d)" % rc)
        self.n_patch = L.orc_n_patch(C.byref(s))
        self.n_macro = L.orc_n_macro(C.byref(s))
        self.mx, self.my = s.m_xi, s.m_eta
        self.nxp = s.n_xi if s.periodic_xi else s.n_xi + 1
        self.nyp = s.n_eta + 1

    # -- pointwise -----------------------------------------------------------
    def map(self, xi, eta):
        o = np.zeros(12)
        self.L.orc_map(C.byref(self.s), float(xi), float(eta), _dp(o))
        return o

    def coeffs(self, xi, eta):
        o = np.zeros(7)
        self.L.orc_coeffs(C.byref(self.s), float(xi), float(eta), _dp(o))
        return o

    def physical(self, x, y):
        o = np.zeros(13)
        self.L.orc_physical(C.byref(self.s), float(x), float(y), _dp(o))
        return o

    def time_factor(self, t):
        return self.L.orc_time_factor(C.byref(self.s), float(t))

    def exact(self, x, y, t):
        return self.L.orc_exact(C.byref(self.s), float(x), float(y), float(t))

    # -- sizes ---------------------------------------------------------------
    def dt_micro(self):
        # a minimum over every micro point of the instance: computed once
        if self._dt_micro is None:
            self._dt_micro = self.L.orc_dt_micro(C.byref(self.s))
        return self._dt_micro

    def dt_macro(self):
        return self.L.orc_dt_macro(C.byref(self.s))

    def tau(self, dt_micro=None):
        return self.s.k_micro * (self.dt_micro() if dt_micro is None else dt_micro)

    # -- fields --------------------------------------------------------------
    def init_field(self, kind=None, params=None, t=0.0):
        kind = self.prob["init"] if kind is None else kind
        params = self.prob["init_p"] if params is None else params
        U = np.zeros(self.n_macro)
        prm = np.array(list(params) + [0.0] * 4, dtype=np.float64)
        self.L.orc_init_field(C.byref(self.s), INIT[kind], _dp(prm), float(t), _dp(U))
        return U

    def micro_coords(self):
        n = self.n_patch * self.mx * self.my
        xi, eta = np.zeros(n), np.zeros(n)
        self.L.orc_micro_coords(C.byref(self.s), _dp(xi), _dp(eta))
        return xi, eta

    def lift(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        u0 = np.zeros(self.n_patch * self.mx * self.my)
        me = max(self.mx, self.my) + 2
        edge = np.zeros(self.n_patch * 4 * me)
        self.L.orc_lift(C.byref(self.s), _dp(U), _dp(u0), _dp(edge))
        return u0.reshape(self.n_patch, self.my, self.mx), edge.reshape(self.n_patch, 4, me)

    def forcing(self, U, t):
        U = np.ascontiguousarray(U, dtype=np.float64)
        r0 = np.zeros(self.n_patch * self.mx * self.my)
        self.L.orc_forcing(C.byref(self.s), _dp(U), float(t), _dp(r0))
        return r0.reshape(self.n_patch, self.my, self.mx)

    def burst(self, U, t, k, dt, form="split"):
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros(self.n_patch * self.mx * self.my)
        self.L.orc_burst(C.byref(self.s), _dp(U), float(t), int(k), float(dt), FORM[form], _dp(out))
        return out.reshape(self.n_patch, self.my, self.mx)

    def restrict(self, U, burst_out, form="split"):
        U = np.ascontiguousarray(U, dtype=np.float64)
        bo = np.ascontiguousarray(burst_out, dtype=np.float64).reshape(-1)
        dU = np.zeros(self.n_patch)
        self.L.orc_restrict(C.byref(self.s), _dp(U), _dp(bo), FORM[form], _dp(dU))
        return dU

    def project(self, U, dU, t, dt_macro, tau):
        U = np.array(U, dtype=np.float64)
        dU = np.ascontiguousarray(dU, dtype=np.float64)
        self.L.orc_project(C.byref(self.s), _dp(U), _dp(dU), float(t), float(dt_macro), float(tau))
        return U

    def apply_bc(self, U, t):
        U = np.array(U, dtype=np.float64)
        self.L.orc_apply_bc(C.byref(self.s), _dp(U), float(t))
        return U

    def step(self, U, t0, dt_macro, n_steps, dt_micro=None, form="split"):
        U = np.array(U, dtype=np.float64)
        dtm = self.dt_micro() if dt_micro is None else dt_micro
        self.L.orc_step(C.byref(self.s), _dp(U), float(t0), float(dt_macro), int(n_steps),
                        float(dtm), FORM[form])
        return U

    def micro_patch(self, p, w0, r, T, K, dt):
        """Split-form micro solve of patch p alone from the departure w0 with
        forcing r (None = 0); returns the departure after K steps."""
        w0 = np.ascontiguousarray(w0, dtype=np.float64).reshape(-1)
        assert w0.size == self.mx * self.my
        out = np.zeros(self.mx * self.my)
        rp = None
        if r is not None:
            r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
            assert r.size == self.mx * self.my
            rp = _dp(r)
        self.L.orc_micro_patch(C.byref(self.s), int(p), _dp(w0), rp, float(T), int(K), float(dt), _dp(out))
        return out.reshape(self.my, self.mx)

    def patch_dU(self, U, t, sel, dt_micro=None, form="split"):
        U = np.ascontiguousarray(U, dtype=np.float64)
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        out = np.zeros(len(sel))
        dtm = self.dt_micro() if dt_micro is None else dt_micro
        self.L.orc_patch_dU(C.byref(self.s), _dp(U), float(t), float(dtm), FORM[form], len(sel),
                            sel.ctypes.data_as(C.POINTER(C.c_int)), _dp(out))
        return out

    def full_domain(self, u, refine, t0, dt, n_steps):
        u = np.array(u, dtype=np.float64)
        self.L.orc_full_domain(C.byref(self.s), int(refine), _dp(u), float(t0), float(dt), int(n_steps))
        return u

    def full_domain_shape(self, refine):
        nx, ny = C.c_int(), C.c_int()
        self.L.orc_full_domain_size(C.byref(self.s), int(refine), C.byref(nx), C.byref(ny))
        return ny.value, nx.value

    # -- indexing helpers ----------------------------------------------------
    def patch_nodes(self):
        """(i, j) macro node of every patch, in patch order."""
        s = self.s
        cols = s.n_xi if s.periodic_xi else s.n_xi - 1
        i0 = 0 if s.periodic_xi else 1
        p = np.arange(self.n_patch)
        return i0 + p % cols, 1 + p // cols

    def node_coords(self):
        """computational coordinates of the macro nodes, shape (nyp, nxp)."""
        s = self.s
        dxi = (s.xi1 - s.xi0) / s.n_xi
        deta = (s.eta1 - s.eta0) / s.n_eta
        xi = s.xi0 + np.arange(self.nxp) * dxi
        eta = s.eta0 + np.arange(self.nyp) * deta
        return np.meshgrid(xi, eta)


def num_threads() -> int:
    """Threads of the oracle's parallel loops over patches."""
    return int(lib().orc_num_threads())


def bessel_root(k, ra, rb, which=1):
    return lib().orc_bessel_root(int(k), float(ra), float(rb), int(which))


def bessel_Z(k, mu, ra, r):
    return lib().orc_bessel_Z(int(k), float(mu), float(ra), float(r))


def bessel_norm(mu, ra, rb, n_int=4000):
    return lib().orc_bessel_norm(float(mu), float(ra), float(rb), int(n_int))


def annulus_series(ra, rb, r, theta, t, n_roots=40):
    return lib().orc_annulus_series(float(ra), float(rb), float(r), float(theta), float(t), int(n_roots))
