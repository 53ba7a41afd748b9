"""Thin Python binding of libpd: torch tensors for device memory, torch's
current CUDA stream for ordering, and argument marshalling to the C ABI.  Every
step of the patch-dynamics path runs in the library's kernels; there is no CPU
or PyTorch fallback."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import _native as N


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libpd needs a CUDA device (GB300, sm_103a)")


def grid_desc(p: dict, prec: str) -> N.GridDesc:
    d = N.GridDesc()
    d.n_xi, d.n_eta, d.periodic_xi = int(p["n_xi"]), int(p["n_eta"]), int(p["periodic_xi"])
    d.xi0, d.xi1, d.eta0, d.eta1 = [float(v) for v in p["box"]]
    d.map = N.MAPS[p["map"]]
    for k in range(4):
        d.map_p[k] = float(p["map_p"][k])
    d.m_xi, d.m_eta = int(p["m_xi"]), int(p["m_eta"])
    d.h_ratio_xi, d.h_ratio_eta = float(p["h_ratio_xi"]), float(p["h_ratio_eta"])
    d.k_micro, d.cfl_micro = int(p["k_micro"]), float(p["cfl_micro"])
    d.prec = N.PD_FP32 if prec == "fp32" else N.PD_FP64
    d.conv_scheme = N.CONV[p["conv"]]
    d.restrict_mode = N.RESTRICT[p["restrict"]]
    d.micro_solver = N.MICRO[p.get("micro", "fe")]
    d.dt_micro = float(p.get("dt_micro") or 0.0)
    return d


def coeff_desc(p: dict):
    c = N.CoeffDesc()
    c.M11, c.M12, c.M22 = [float(v) for v in p["M"]]
    c.d0, c.dx, c.dy = [float(v) for v in p["d_aff"]]
    c.ds, c.dk = [float(v) for v in p["d_sin"]]
    four = p["four"]
    c.n_four = len(four["c"])
    for k in range(c.n_four):
        c.four_c[k] = float(four["c"][k])
        c.four_phi[k] = float(four["phi"][k])
    c.four_ra, c.four_rb = float(four["ra"]), float(four["rb"])
    for k in range(3):
        c.va[k] = float(p["va"][k])
        c.vb[k] = float(p["vb"][k])
        c.src_p[k] = float(p["src_p"][k])
    c.f0 = float(p["f0"])
    c.src = N.SRC[p["src"]]
    amp = None
    if p.get("src_amp") is not None:
        amp = np.ascontiguousarray(p["src_amp"], dtype=np.float64)
        c.src_amp = amp.ctypes.data_as(C.POINTER(C.c_double))
    c.tkind, c.tc = N.TIME[p["time"]], float(p["tc"])
    c.sol = N.SOL[p["sol"]]
    return c, amp


def _ptr(t: torch.Tensor) -> int:
    assert t.is_cuda and t.is_contiguous()
    return t.data_ptr()


class Grid:
    """A set of patch-dynamics instances on the current CUDA device.

    probs: one workloads-style problem dictionary or a list of them (all with
    the same micro size and precision).  prec: "fp32" (FP32 bursts, FP64
    restriction and projection) or "fp64"."""

    def __init__(self, probs, prec: str = "fp32", graphs: bool = True, persistent: bool | None = None,
                 storage: str = "auto", autotune: bool = True, integrator: str = "euler"):
        """persistent: None follows the PD_PERSISTENT environment variable (default on;
        "0" selects one fused launch per macro step, e.g. for kernel profilers that
        cannot replay cooperative launches)."""
        _require_cuda()
        if persistent is None:
            persistent = os.environ.get("PD_PERSISTENT", "1") != "0"
        self.L = N.load()
        if isinstance(probs, dict):
            probs = [probs]
        self.probs = [dict(p) for p in probs]
        self.prec = prec
        self.device = torch.device("cuda", torch.cuda.current_device())
        n = len(self.probs)
        descs = (N.GridDesc * n)(*[grid_desc(p, prec) for p in self.probs])
        h = C.c_void_p()
        st = torch.cuda.current_stream().cuda_stream
        rc = self.L.pd_create_grid(descs, n, C.c_void_p(st), C.byref(h))
        if rc != N.PD_OK:
            raise N.PDError(rc, "pd_create_grid rejected the descriptors")
        self.h = h
        self.L.pd_set_graph_mode(self.h, 1 if graphs else 0)
        self.L.pd_set_persistent(self.h, 1 if persistent else 0)
        N.check(self.L.pd_set_integrator(self.h, N.INTEGRATORS[integrator]), self.h)
        q = {int(p.get("q_refresh") or 1) for p in self.probs}
        if len(q) != 1:
            raise ValueError("all instances of a grid share one edge-refresh count")
        N.check(self.L.pd_set_edge_refresh(self.h, q.pop()), self.h)
        N.check(self.L.pd_set_coeff_storage(self.h, {"auto": 0, "records": 1, "tables": 2}[storage]), self.h)
        if not autotune:
            N.check(self.L.pd_set_autotune(self.h, 0, 128, 0), self.h)
        for k, p in enumerate(self.probs):
            c, amp = coeff_desc(p)
            N.check(self.L.pd_set_coeffs(self.h, k, C.byref(c)), self.h)
            del amp
        nm, npch, sb = C.c_longlong(), C.c_longlong(), C.c_size_t()
        N.check(self.L.pd_sizes(self.h, C.byref(nm), C.byref(npch), C.byref(sb)), self.h)
        self.n_macro_total, self.n_patch_total, self.state_bytes = nm.value, npch.value, sb.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.L.pd_destroy_grid(h)
            except Exception:
                pass
            self.h = C.c_void_p()

    # -- plumbing -------------------------------------------------------------
    def _stream(self):
        self.L.pd_set_stream(self.h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def info(self, inst: int = 0) -> dict:
        o = N.Info()
        N.check(self.L.pd_query(self.h, inst, C.byref(o)), self.h)
        return {f: getattr(o, f) for f, _ in N.Info._fields_}

    def new_field(self) -> torch.Tensor:
        return torch.zeros(self.n_macro_total, dtype=torch.float64, device=self.device)

    def new_state(self) -> torch.Tensor:
        return torch.zeros(self.state_bytes, dtype=torch.uint8, device=self.device)

    def state_views(self, state: torch.Tensor, inst: int = 0) -> dict:
        """typed views of instance `inst`'s parts of the micro-state sections."""
        i = self.info(inst)
        P, mx, my, es = i["n_patch"], i["m_xi"], i["m_eta"], i["edge_stride"]
        rdt = torch.float32 if self.prec == "fp32" else torch.float64
        rb = 4 if self.prec == "fp32" else 8

        def sec(off, start, n, dt, b):
            o = off + start * b
            return state[o:o + n * b].view(dt)
        pt, eo, po = i["point_offset"], i["edge_offset"], i["patch_offset"]
        return {
            "u0": sec(i["off_u0"], pt, P * mx * my, torch.float64, 8).view(P, my, mx),
            "r": sec(i["off_r"], pt, P * mx * my, rdt, rb).view(P, my, mx),
            "w": sec(i["off_w"], pt, P * mx * my, rdt, rb).view(P, my, mx),
            "edge": sec(i["off_edge"], eo, P * 4 * es, torch.float64, 8).view(P, 4, es),
            "bias": sec(i["off_bias"], po, P, torch.float64, 8),
        }

    # -- C-ABI entry points ----------------------------------------------------
    def init_field(self, U: torch.Tensor | None = None, t: float = 0.0, kinds=None) -> torch.Tensor:
        U = self.new_field() if U is None else U
        self._stream()
        for k, p in enumerate(self.probs):
            kind = p["init"] if kinds is None else kinds[k]
            prm = list(p.get("init_p", [])) or [0.0]
            arr = (C.c_double * len(prm))(*prm)
            N.check(self.L.pd_init_field(self.h, k, N.INIT[kind], arr, len(prm), float(t),
                                         C.c_void_p(_ptr(U))), self.h)
        return U

    def coeffs(self, inst: int = 0) -> torch.Tensor:
        i = self.info(inst)
        out = torch.empty(i["n_patch"] * i["m_xi"] * i["m_eta"] * 8, dtype=torch.float64, device=self.device)
        self._stream()
        N.check(self.L.pd_get_coeffs(self.h, inst, C.c_void_p(_ptr(out))), self.h)
        return out.view(i["n_patch"], i["m_eta"], i["m_xi"], 8)

    def lift(self, U: torch.Tensor, t: float, state: torch.Tensor):
        self._stream()
        N.check(self.L.pd_lift(self.h, C.c_void_p(_ptr(U)), float(t), C.c_void_p(_ptr(state))), self.h)

    def micro_burst(self, state: torch.Tensor, t: float, k_steps: int):
        self._stream()
        N.check(self.L.pd_micro_burst(self.h, C.c_void_p(_ptr(state)), float(t), int(k_steps)), self.h)

    def restrict(self, state: torch.Tensor, dU: torch.Tensor | None = None) -> torch.Tensor:
        dU = torch.empty(self.n_patch_total, dtype=torch.float64, device=self.device) if dU is None else dU
        self._stream()
        N.check(self.L.pd_restrict(self.h, C.c_void_p(_ptr(state)), C.c_void_p(_ptr(dU))), self.h)
        return dU

    def project(self, U: torch.Tensor, dU: torch.Tensor, t: float, dt_macro: float):
        self._stream()
        N.check(self.L.pd_project(self.h, C.c_void_p(_ptr(U)), C.c_void_p(_ptr(dU)), float(t),
                                  float(dt_macro)), self.h)

    def step(self, U: torch.Tensor, t0: float, dt_macro: float, n_macro: int):
        self._stream()
        N.check(self.L.pd_step(self.h, C.c_void_p(_ptr(U)), float(t0), float(dt_macro), int(n_macro)), self.h)

    def step_noalloc(self, U: torch.Tensor, t0: float, dt_macro: float, n_macro: int):
        """pd_step_noalloc: the per-step fused path with fixed library scratch."""
        self._stream()
        N.check(self.L.pd_step_noalloc(self.h, C.c_void_p(_ptr(U)), float(t0), float(dt_macro), int(n_macro)), self.h)

    def sync(self):
        N.check(self.L.pd_sync(self.h), self.h)

    def launches(self) -> int:
        return int(self.L.pd_launch_count(self.h))

    def autotune(self, n_trial_steps: int = 2):
        b, h = C.c_int(), C.c_int()
        N.check(self.L.pd_autotune(self.h, int(n_trial_steps), C.byref(b), C.byref(h)), self.h)
        return b.value, bool(h.value)

    def set_wait_limit(self, ns: int):
        N.check(self.L.pd_set_wait_limit(self.h, int(ns)), self.h)

    def silence_warp(self, warp: int):
        """test hook: item warp `warp` of the persistent kernel never publishes"""
        N.check(self.L.pd_test_silence_warp(self.h, int(warp)), self.h)

    def set_timing(self, enabled: bool):
        N.check(self.L.pd_set_timing(self.h, 1 if enabled else 0), self.h)

    def timing(self):
        """(summed fused-kernel event time in ms, fused launches covered)"""
        ms, n = C.c_double(), C.c_longlong()
        N.check(self.L.pd_get_timing(self.h, C.byref(ms), C.byref(n)), self.h)
        return ms.value, n.value

    def save_checkpoint(self, U: torch.Tensor, t: float, step: int, path: str):
        self._stream()
        N.check(self.L.pd_save_checkpoint(self.h, C.c_void_p(_ptr(U)), float(t), int(step),
                                          path.encode()), self.h)

    def load_checkpoint(self, U: torch.Tensor, path: str):
        t, s = C.c_double(), C.c_longlong()
        self._stream()
        N.check(self.L.pd_load_checkpoint(self.h, C.c_void_p(_ptr(U)), C.byref(t), C.byref(s),
                                          path.encode()), self.h)
        return t.value, s.value


class MLP:
    """The surrogate network of include/pd_surrogate.h on the current CUDA
    device (35 -> 256 -> 256 -> 256 -> 1, BF16 tensor-core GEMMs).  Inputs
    are BF16 tensors [n, 128] (high parts, then low parts); parameters are a
    flat FP32 vector."""

    N_PARAM = N.MLP_N_PARAM

    def __init__(self, max_batch: int = 8192):
        if not torch.cuda.is_available():
            raise RuntimeError("the surrogate network needs a CUDA device")
        self.L = N.load()
        h = C.c_void_p()
        N.check_mlp(self.L.pd_mlp_create(int(max_batch), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         C.byref(h)))
        self.h = h
        self.max_batch = int(max_batch)

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.pd_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def _stream(self):
        self.L.pd_mlp_set_stream(self.h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def _chk(self, rc):
        N.check_mlp(rc, self.h)

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        self._stream()
        self._chk(self.L.pd_mlp_set_params(self.h, th.ctypes.data_as(C.POINTER(C.c_float)), th.size))

    def init(self, seed: int):
        """fan-in uniform initialisation on the device"""
        self._stream()
        self._chk(self.L.pd_mlp_init(self.h, int(seed)))

    def params(self) -> np.ndarray:
        th = np.zeros(self.N_PARAM, dtype=np.float32)
        self._stream()
        self._chk(self.L.pd_mlp_get_params(self.h, th.ctypes.data_as(C.POINTER(C.c_float)), th.size))
        return th

    def set_norm(self, mu, sigma, y_scale: float):
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sg = np.ascontiguousarray(sigma, dtype=np.float32)
        self._stream()
        self._chk(self.L.pd_mlp_set_norm(self.h, mu.ctypes.data_as(C.POINTER(C.c_float)),
                                         sg.ctypes.data_as(C.POINTER(C.c_float)), float(y_scale)))

    def norm(self):
        mu = np.zeros(N.MLP_N_IN, dtype=np.float32)
        sg = np.zeros(N.MLP_N_IN, dtype=np.float32)
        ys = C.c_float()
        self._chk(self.L.pd_mlp_get_norm(self.h, mu.ctypes.data_as(C.POINTER(C.c_float)),
                                         sg.ctypes.data_as(C.POINTER(C.c_float)), C.byref(ys)))
        return mu, sg, ys.value

    def fit_norm(self, X_raw: torch.Tensor, y_raw: torch.Tensor):
        self._stream()
        self._chk(self.L.pd_mlp_fit_norm(self.h, C.c_void_p(_ptr(X_raw)), C.c_void_p(_ptr(y_raw)), X_raw.shape[0]))

    def pack(self, X_raw: torch.Tensor, y_raw: torch.Tensor = None):
        n = X_raw.shape[0]
        X = torch.empty((n, N.MLP_IN_COLS), dtype=torch.bfloat16, device=X_raw.device)
        t = torch.empty(n, dtype=torch.float32, device=X_raw.device) if y_raw is not None else None
        self._stream()
        self._chk(self.L.pd_mlp_pack(self.h, C.c_void_p(_ptr(X_raw)),
                                     C.c_void_p(_ptr(y_raw)) if y_raw is not None else None, n,
                                     C.c_void_p(_ptr(X)), C.c_void_p(_ptr(t)) if t is not None else None))
        return X, t

    def forward(self, X: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device) if out is None else out
        self._stream()
        self._chk(self.L.pd_mlp_forward(self.h, C.c_void_p(_ptr(X)), X.shape[0], C.c_void_p(_ptr(y))))
        return y

    def gradient(self, X: torch.Tensor, t: torch.Tensor):
        g = torch.empty(self.N_PARAM, dtype=torch.float32, device=X.device)
        loss = C.c_float()
        self._stream()
        self._chk(self.L.pd_mlp_gradient(self.h, C.c_void_p(_ptr(X)), C.c_void_p(_ptr(t)), X.shape[0],
                                         C.c_void_p(_ptr(g)), C.byref(loss)))
        return g, loss.value

    def adam_step(self, lr: float):
        self._stream()
        self._chk(self.L.pd_mlp_adam_step(self.h, float(lr)))

    def train(self, X: torch.Tensor, t: torch.Tensor, batch: int, epochs: int, lr_max: float, seed: int = 0):
        hist = np.zeros(max(epochs, 1), dtype=np.float32)
        self._stream()
        self._chk(self.L.pd_mlp_train(self.h, C.c_void_p(_ptr(X)), C.c_void_p(_ptr(t)), X.shape[0], int(batch),
                                      int(epochs), float(lr_max), int(seed),
                                      hist.ctypes.data_as(C.POINTER(C.c_float))))
        return hist[:epochs]

    def sync(self):
        self._chk(self.L.pd_mlp_sync(self.h))


class Surrogate:
    """The surrogate on a one-instance Grid (include/pd_surrogate.h): features,
    training targets from the patch solver, and macro steps with the residual
    check and the burst fallback."""

    def __init__(self, grid: Grid, net: MLP):
        self.grid, self.net = grid, net
        self.L = N.load()
        grid._stream()
        net._stream()
        h = C.c_void_p()
        N.check(self.L.pd_surrogate_create(grid.h, net.h, C.byref(h)), grid.h)
        self.h = h
        self.n_patch = grid.info(0)["n_patch"]

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.pd_surrogate_destroy(self.h)
            self.h = C.c_void_p()

    def _pre(self):
        self.grid._stream()
        self.net._stream()

    def _p(self, t):
        return C.c_void_p(_ptr(t)) if t is not None else None

    def features(self, U: torch.Tensor, standardised: bool = True, raw: bool = False):
        n = self.n_patch
        X = torch.empty((n, N.MLP_IN_COLS), dtype=torch.bfloat16, device=U.device) if standardised else None
        scale = torch.empty(n, dtype=torch.float64, device=U.device) if standardised else None
        Xr = torch.empty((n, N.MLP_N_IN), dtype=torch.float32, device=U.device) if raw else None
        Rs = torch.empty(n, dtype=torch.float64, device=U.device) if raw else None
        self._pre()
        N.check(self.L.pd_surrogate_features(self.h, self._p(U), self._p(X), self._p(scale), self._p(Xr), self._p(Rs)),
                self.grid.h)
        return dict(X=X, scale=scale, X_raw=Xr, Rs=Rs)

    def targets(self, U: torch.Tensor, t: float, Rs: torch.Tensor) -> torch.Tensor:
        y = torch.empty(self.n_patch, dtype=torch.float32, device=U.device)
        self._pre()
        N.check(self.L.pd_surrogate_targets(self.h, self._p(U), float(t), self._p(Rs), self._p(y)), self.grid.h)
        return y

    def evaluate(self, U: torch.Tensor, t: float, F_hat=True, F1=True, F=True):
        out = {k: (torch.empty(self.n_patch, dtype=torch.float64, device=U.device) if want else None)
               for k, want in (("F_hat", F_hat), ("F1", F1), ("F", F))}
        self._pre()
        N.check(self.L.pd_surrogate_evaluate(self.h, self._p(U), float(t), self._p(out["F_hat"]), self._p(out["F1"]),
                                             self._p(out["F"])), self.grid.h)
        return out

    def step(self, U: torch.Tensor, t0: float, dt_macro: float, n_macro: int, eps: float = 1e-3):
        self._pre()
        N.check(self.L.pd_surrogate_step(self.h, self._p(U), float(t0), float(dt_macro), int(n_macro), float(eps)),
                self.grid.h)

    def step_f1(self, U: torch.Tensor, t0: float, dt_macro: float, n_macro: int):
        """The same macro steps with every patch's F taken from the one-micro-step
        estimate F1 (no network)."""
        self._pre()
        N.check(self.L.pd_surrogate_step_f1(self.h, self._p(U), float(t0), float(dt_macro), int(n_macro)),
                self.grid.h)

    def perturb(self, U: torch.Tensor, rel_sigma: float, seed: int, out: torch.Tensor = None) -> torch.Tensor:
        """U plus seeded grid-scale noise of relative size rel_sigma on the interior nodes"""
        V = torch.empty_like(U) if out is None else out
        self._pre()
        N.check(self.L.pd_surrogate_perturb(self.h, self._p(U), float(rel_sigma), int(seed), self._p(V)), self.grid.h)
        return V

    def counts(self):
        a, b = C.c_longlong(), C.c_longlong()
        N.check(self.L.pd_surrogate_counts(self.h, C.byref(a), C.byref(b)), self.grid.h)
        return a.value, b.value
