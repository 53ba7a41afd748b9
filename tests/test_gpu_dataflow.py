"""The persistent dataflow execution of pd_step: identical results to one fused
launch per macro step, multi-chunk runs, and the bounded-wait failure path
(a producer that never publishes makes its neighbours give up; the host sees
PD_ETIMEOUT and the context stays usable).  No GPU fault is involved."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "c2s": W.c2_heterogeneous(n=20, m=11, n_macro=16),
    "c3s": W.c3_annulus(n_r=13, n_theta=30, m=9),
    "p411": W.paper_cdr(False, lam=0.1, n=12, m=11),
    "macro_m5": dict(W.c1_manufactured(n=11, m=5), restrict="macro"),
    "polar_cross_m7": W.base(n_xi=17, n_eta=7, periodic_xi=1, box=(0, 2 * math.pi, 0, 1), map="polar",
                             map_p=(0.8, 2.2, 1.0, 0), m_xi=7, m_eta=7, M=(1.0, 0.2, 0.5),
                             va=(0.3, 0.0, 0.0), vb=(0.0, 0.0, 0.2), f0=0.4, init="bump"),
}


@pytest.fixture(scope="module")
def Grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_08764_gb300.api import Grid
    return Grid


def _run(Grid, p, prec, persistent, n, dtm=None):
    g = Grid(p, prec=prec, persistent=persistent)
    dtm = 0.5 * g.info()["dt_macro_suggested"] if dtm is None else dtm
    U = g.init_field()
    g.step(U, 0.1, dtm, n)
    g.sync()
    return U.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_persistent_equals_per_step_launches(Grid, name, prec):
    p = CASES[name]
    a = _run(Grid, p, prec, True, 9)
    b = _run(Grid, p, prec, False, 9)
    scale = np.abs(b).max()
    assert np.abs(a - b).max() <= 1e-13 * scale, (name, prec, np.abs(a - b).max() / scale)


def test_multi_chunk_run_equals_per_step_launches(Grid):
    """FP64 with a time-dependent source: the step count exceeds one
    persistent chunk, so several cooperative launches share the flags."""
    p = W.paper_cdr(True, lam=0.2, n=9, m=7)
    a = _run(Grid, p, "fp64", True, 420, dtm=1e-5)
    b = _run(Grid, p, "fp64", False, 420, dtm=1e-5)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_silent_producer_times_out_and_the_grid_recovers(Grid):
    from paper_2405_08764_gb300 import _native as N
    p = CASES["c2s"]
    g = Grid(p, prec="fp32", persistent=True)
    g.set_wait_limit(50_000_000)          # 50 ms
    g.silence_warp(5)
    U = g.init_field()
    g.step(U, 0.0, 1e-5, 6)
    with pytest.raises(N.PDError) as e:
        g.sync()
    assert e.value.status == N.PD_ETIMEOUT
    # the context is intact: normal operation afterwards matches a fresh grid
    g.silence_warp(-1)
    g.set_wait_limit(250_000_000)
    V = g.init_field()
    g.step(V, 0.1, 1e-5, 6)
    g.sync()
    ref = _run(Grid, p, "fp32", False, 6, dtm=1e-5)
    assert np.abs(V.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
