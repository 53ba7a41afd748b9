"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every function the headers in include/ declare (no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    import glob
    names = set()
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(pd_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2405_08764_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("pd_create_grid", "pd_set_coeffs", "pd_lift", "pd_micro_burst", "pd_restrict",
                 "pd_project", "pd_step", "pd_destroy_grid"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_status_strings(lib):
    lib.pd_abi_version.restype = ctypes.c_int
    assert lib.pd_abi_version() == 2
    lib.pd_status_str.restype = ctypes.c_char_p
    lib.pd_status_str.argtypes = [ctypes.c_int]
    assert lib.pd_status_str(0) == b"ok"
    assert b"invalid" in lib.pd_status_str(1)


def test_create_rejects_bad_descriptors_before_touching_the_device(lib):
    from paper_2405_08764_gb300 import _native as N
    from paper_2405_08764_gb300.api import grid_desc
    from paper_2405_08764_gb300 import workloads as W
    L = N.load()
    for bad in (dict(m_xi=2), dict(h_ratio_xi=1.0), dict(k_micro=0), dict(n_xi=1), dict(cfl_micro=1.5),
                dict(map="polar", map_p=(2.0, 1.0, 0, 0))):
        p = W.base(**bad)
        d = grid_desc(p, "fp32")
        h = ctypes.c_void_p()
        rc = L.pd_create_grid(ctypes.byref(d), 1, None, ctypes.byref(h))
        assert rc == N.PD_EINVAL, bad


def _create(L, descs, n=None, out=True):
    arr = (type(descs[0]) * len(descs))(*descs)
    h = ctypes.c_void_p()
    return L.pd_create_grid(arr, len(descs) if n is None else n, None, ctypes.byref(h) if out else None)


def test_create_rejects_every_invalid_field_and_combination(lib):
    """Each validation branch of pd_create_grid returns PD_EINVAL on the host,
    before any device allocation (this machine has no GPU)."""
    from paper_2405_08764_gb300 import _native as N
    from paper_2405_08764_gb300.api import grid_desc
    from paper_2405_08764_gb300 import workloads as W
    L = N.load()
    ok = W.base()
    bad_dicts = [dict(m_xi=33), dict(m_eta=2), dict(k_micro=4097), dict(h_ratio_eta=0.0), dict(h_ratio_xi=-0.1),
                 dict(n_eta=1), dict(periodic_xi=1, n_xi=2), dict(micro="adi", m_xi=13, m_eta=13, dt_micro=1e-6),
                 dict(micro="adi", m_xi=7, m_eta=9, dt_micro=1e-6), dict(dt_micro=-1e-6),
                 dict(dt_micro=float("inf")), dict(cfl_micro=0.0), dict(box=(1.0, 1.0, 0.0, 1.0)),
                 dict(box=(0.0, 1.0, 0.5, 0.2)), dict(map="sine", map_p=(1.0, 0, 0, 0)),
                 dict(map="polar", map_p=(0.0, 1.0, 0, 0))]
    for bad in bad_dicts:
        assert _create(L, [grid_desc(W.base(**bad), "fp32")]) == N.PD_EINVAL, bad
    for field, value in (("map", 7), ("prec", 5), ("conv_scheme", 3), ("restrict_mode", -1), ("micro_solver", 9)):
        d = grid_desc(ok, "fp32")
        setattr(d, field, value)
        assert _create(L, [d]) == N.PD_EINVAL, field
    # mixed precisions, and the ADI solver on a grid of several instances
    assert _create(L, [grid_desc(ok, "fp32"), grid_desc(ok, "fp64")]) == N.PD_EINVAL
    adi = dict(ok, micro="adi", dt_micro=1e-6)
    assert _create(L, [grid_desc(adi, "fp32"), grid_desc(adi, "fp32")]) == N.PD_EINVAL
    # no instances, no output pointer, no descriptors
    assert _create(L, [grid_desc(ok, "fp32")], n=0) == N.PD_EINVAL
    assert _create(L, [grid_desc(ok, "fp32")], out=False) == N.PD_EINVAL
    h = ctypes.c_void_p()
    assert L.pd_create_grid(None, 1, None, ctypes.byref(h)) == N.PD_EINVAL


def test_calls_on_a_null_grid_are_rejected(lib):
    from paper_2405_08764_gb300 import _native as N
    L = N.load()
    for name, args in (("pd_step", (None, None, ctypes.c_double(0.0), ctypes.c_double(1e-3), 1)),
                       ("pd_sync", (None,)), ("pd_set_edge_refresh", (None, 2)), ("pd_set_integrator", (None, 1))):
        assert getattr(L, name)(*args) == N.PD_EINVAL, name


def test_binding_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2405_08764_gb300.api import Grid
    from paper_2405_08764_gb300 import workloads as W
    with pytest.raises(RuntimeError):
        Grid(W.c1_manufactured())


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2405_08764_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "pd_oracle" not in txt, f
