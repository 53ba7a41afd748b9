"""ctypes declarations of the C ABI in include/pd.h and include/pd_surrogate.h
(argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PD_LIB_PATH") or os.path.join(HERE, "libpd.so")

PD_OK, PD_EINVAL, PD_ENOMEM, PD_ECUDA, PD_ESTATE, PD_EUNSTABLE, PD_ETIMEOUT, PD_ENUMERIC = range(8)
PD_FP64, PD_FP32 = 0, 1
INTEGRATORS = {"euler": 0, "heun": 1, "ab2": 2}

MAPS = {"identity": 0, "sine": 1, "tanh": 2, "polar": 3}
CONV = {"upwind": 0, "central": 1}
RESTRICT = {"lifted": 0, "macro": 1}
MICRO = {"fe": 0, "adi": 1}
SRC = {"none": 0, "mms_sinprod": 1, "exp_linear": 2, "gauss_patch": 3}
TIME = {"const": 0, "exp": 1, "sin": 2}
SOL = {"none": 0, "exp_xyt": 1, "sinprod_decay": 2}
INIT = {"zero": 0, "exact": 1, "bessel": 2, "bump": 3, "annulus_poly": 4}


class GridDesc(C.Structure):
    _fields_ = [
        ("n_xi", C.c_int), ("n_eta", C.c_int), ("periodic_xi", C.c_int),
        ("xi0", C.c_double), ("xi1", C.c_double), ("eta0", C.c_double), ("eta1", C.c_double),
        ("map", C.c_int), ("map_p", C.c_double * 4),
        ("m_xi", C.c_int), ("m_eta", C.c_int),
        ("h_ratio_xi", C.c_double), ("h_ratio_eta", C.c_double),
        ("k_micro", C.c_int), ("cfl_micro", C.c_double),
        ("prec", C.c_int), ("conv_scheme", C.c_int), ("restrict_mode", C.c_int),
        ("micro_solver", C.c_int), ("dt_micro", C.c_double),
    ]


class CoeffDesc(C.Structure):
    _fields_ = [
        ("M11", C.c_double), ("M12", C.c_double), ("M22", C.c_double),
        ("d0", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("ds", C.c_double), ("dk", C.c_double),
        ("n_four", C.c_int), ("four_c", C.c_double * 3), ("four_phi", C.c_double * 3),
        ("four_ra", C.c_double), ("four_rb", C.c_double),
        ("va", C.c_double * 3), ("vb", C.c_double * 3), ("f0", C.c_double),
        ("src", C.c_int), ("src_p", C.c_double * 3), ("src_amp", C.POINTER(C.c_double)),
        ("tkind", C.c_int), ("tc", C.c_double),
        ("sol", C.c_int),
    ]


class Info(C.Structure):
    _fields_ = [
        ("n_patch", C.c_int), ("n_macro", C.c_int), ("nxp", C.c_int), ("nyp", C.c_int),
        ("m_xi", C.c_int), ("m_eta", C.c_int), ("k_micro", C.c_int), ("prec", C.c_int),
        ("u_offset", C.c_longlong), ("patch_offset", C.c_longlong),
        ("point_offset", C.c_longlong), ("edge_offset", C.c_longlong),
        ("dt_micro", C.c_double), ("tau", C.c_double), ("dt_macro_suggested", C.c_double),
        ("state_bytes", C.c_size_t), ("off_u0", C.c_size_t), ("off_r", C.c_size_t),
        ("off_w", C.c_size_t), ("off_edge", C.c_size_t), ("off_bias", C.c_size_t),
        ("edge_stride", C.c_int), ("exec_path", C.c_int), ("chunk_steps", C.c_int),
        ("has_cross", C.c_int), ("has_tsrc", C.c_int),
    ]


_VP = C.c_void_p
_GP = C.c_void_p
SIGNATURES = {
    "pd_create_grid": (C.c_int, [C.POINTER(GridDesc), C.c_int, _VP, C.POINTER(_GP)]),
    "pd_destroy_grid": (C.c_int, [_GP]),
    "pd_set_stream": (C.c_int, [_GP, _VP]),
    "pd_set_coeffs": (C.c_int, [_GP, C.c_int, C.POINTER(CoeffDesc)]),
    "pd_query": (C.c_int, [_GP, C.c_int, C.POINTER(Info)]),
    "pd_sizes": (C.c_int, [_GP, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_size_t)]),
    "pd_get_coeffs": (C.c_int, [_GP, C.c_int, _VP]),
    "pd_init_field": (C.c_int, [_GP, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double, _VP]),
    "pd_lift": (C.c_int, [_GP, _VP, C.c_double, _VP]),
    "pd_micro_burst": (C.c_int, [_GP, _VP, C.c_double, C.c_int]),
    "pd_restrict": (C.c_int, [_GP, _VP, _VP]),
    "pd_project": (C.c_int, [_GP, _VP, _VP, C.c_double, C.c_double]),
    "pd_step": (C.c_int, [_GP, _VP, C.c_double, C.c_double, C.c_int]),
    "pd_step_noalloc": (C.c_int, [_GP, _VP, C.c_double, C.c_double, C.c_int]),
    "pd_set_graph_mode": (C.c_int, [_GP, C.c_int]),
    "pd_set_persistent": (C.c_int, [_GP, C.c_int]),
    "pd_set_integrator": (C.c_int, [_GP, C.c_int]),
    "pd_set_edge_refresh": (C.c_int, [_GP, C.c_int]),
    "pd_set_coeff_storage": (C.c_int, [_GP, C.c_int]),
    "pd_autotune": (C.c_int, [_GP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pd_set_autotune": (C.c_int, [_GP, C.c_int, C.c_int, C.c_int]),
    "pd_set_wait_limit": (C.c_int, [_GP, C.c_longlong]),
    "pd_test_silence_warp": (C.c_int, [_GP, C.c_int]),
    "pd_sync": (C.c_int, [_GP]),
    "pd_save_checkpoint": (C.c_int, [_GP, _VP, C.c_double, C.c_longlong, C.c_char_p]),
    "pd_load_checkpoint": (C.c_int, [_GP, _VP, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_char_p]),
    "pd_launch_count": (C.c_longlong, [_GP]),
    "pd_set_timing": (C.c_int, [_GP, C.c_int]),
    "pd_get_timing": (C.c_int, [_GP, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "pd_status_str": (C.c_char_p, [C.c_int]),
    "pd_last_error": (C.c_char_p, [_GP]),
    "pd_abi_version": (C.c_int, []),
    # learned surrogate (include/pd_surrogate.h)
    "pd_mlp_create": (C.c_int, [C.c_int, _VP, C.POINTER(_VP)]),
    "pd_mlp_destroy": (C.c_int, [_VP]),
    "pd_mlp_set_stream": (C.c_int, [_VP, _VP]),
    "pd_mlp_set_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.c_int]),
    "pd_mlp_get_params": (C.c_int, [_VP, C.POINTER(C.c_float), C.c_int]),
    "pd_mlp_init": (C.c_int, [_VP, C.c_ulonglong]),
    "pd_mlp_set_norm": (C.c_int, [_VP, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float]),
    "pd_mlp_get_norm": (C.c_int, [_VP, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "pd_mlp_fit_norm": (C.c_int, [_VP, _VP, _VP, C.c_longlong]),
    "pd_mlp_pack": (C.c_int, [_VP, _VP, _VP, C.c_longlong, _VP, _VP]),
    "pd_mlp_forward": (C.c_int, [_VP, _VP, C.c_longlong, _VP]),
    "pd_mlp_gradient": (C.c_int, [_VP, _VP, _VP, C.c_int, _VP, C.POINTER(C.c_float)]),
    "pd_mlp_train": (C.c_int, [_VP, _VP, _VP, C.c_longlong, C.c_int, C.c_int, C.c_float, C.c_ulonglong,
                               C.POINTER(C.c_float)]),
    "pd_mlp_adam_step": (C.c_int, [_VP, C.c_float]),
    "pd_mlp_sync": (C.c_int, [_VP]),
    "pd_mlp_last_error": (C.c_char_p, [_VP]),
    "pd_surrogate_create": (C.c_int, [_GP, _VP, C.POINTER(_VP)]),
    "pd_surrogate_destroy": (C.c_int, [_VP]),
    "pd_surrogate_features": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "pd_surrogate_targets": (C.c_int, [_VP, _VP, C.c_double, _VP, _VP]),
    "pd_surrogate_evaluate": (C.c_int, [_VP, _VP, C.c_double, _VP, _VP, _VP]),
    "pd_surrogate_step": (C.c_int, [_VP, _VP, C.c_double, C.c_double, C.c_int, C.c_double]),
    "pd_surrogate_step_f1": (C.c_int, [_VP, _VP, C.c_double, C.c_double, C.c_int]),
    "pd_surrogate_counts": (C.c_int, [_VP, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "pd_surrogate_perturb": (C.c_int, [_VP, _VP, C.c_double, C.c_ulonglong, _VP]),
}
MLP_N_IN, MLP_N_PAD, MLP_IN_COLS, MLP_WIDTH, MLP_N_PARAM = 35, 64, 128, 256, 148481

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libpd.so; raises if the CUDA library has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError("libpd.so not found at %s: build it with "
                                   "`python -m paper_2405_08764_gb300.build`" % path)
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class PDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (load().pd_status_str(status).decode(), status, msg))
        self.status = status


def check(status: int, grid=None):
    if status != PD_OK:
        msg = load().pd_last_error(grid).decode() if grid else ""
        raise PDError(status, msg)


def check_mlp(status: int, net=None):
    if status != PD_OK:
        msg = load().pd_mlp_last_error(net).decode() if net else ""
        raise PDError(status, msg)
