"""pd_step_noalloc (fused per-step path with its scratch in a fixed library
array) against pd_step on the same grid description, over two calls in a row.
Named to be collected last: it also has to pass after every other GPU test has
used the library in the same process."""
import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "c2_m11": W.c2_heterogeneous(n=24, m=11, n_macro=16),
    "c1_m7": W.c1_manufactured(n=12, m=7),
    "annulus_m9": W.c3_annulus(n_r=11, n_theta=26, m=9),
    # Section 4.1 with the paper's ADI bursts (two nano steps per burst)
    "paper411_adi": W.paper_cdr_adi(False, 0.1, 10, 2000),
}


@pytest.fixture(scope="module")
def Grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_08764_gb300.api import Grid
    return Grid


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_two_calls_match_pd_step(Grid, name, prec):
    p = CASES[name]
    ref = Grid(p, prec=prec, persistent=False)
    mine = Grid(p, prec=prec, persistent=False)
    dtm = 0.5 * ref.info()["dt_macro_suggested"]
    U, V = ref.init_field(), mine.init_field()
    # odd then even step counts: the result ends in the fixed array once and in U once
    for t0, n in ((0.0, 5), (5 * dtm, 4)):
        ref.step(U, t0, dtm, n)
        mine.step_noalloc(V, t0, dtm, n)
        ref.sync()
        mine.sync()
        a, b = V.cpu().numpy(), U.cpu().numpy()
        assert np.isfinite(a).all()
        # same kernels and arithmetic as pd_step's per-step path
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (name, prec, t0)


def test_rejects_requests_beyond_the_fixed_array(Grid):
    from paper_2405_08764_gb300 import _native as N
    g = Grid(CASES["c1_m7"], prec="fp64", persistent=False)
    U = g.init_field()
    before = U.clone()
    k = g.info()["k_micro"]
    too_many = (1 << 19) // (k + 3) + 1
    with pytest.raises(N.PDError) as e:
        g.step_noalloc(U, 0.0, 0.0, too_many)
    assert e.value.status == N.PD_EINVAL
    g.sync()
    assert torch.equal(U, before)
    # a grid of several instances is refused too
    h = Grid([CASES["c1_m7"], CASES["c1_m7"]], prec="fp64")
    W2 = h.init_field()
    with pytest.raises(N.PDError) as e:
        h.step_noalloc(W2, 0.0, 0.0, 1)
    assert e.value.status == N.PD_EINVAL


@pytest.mark.parametrize("setting", ["heun", "ab2", "q_refresh"])
def test_refuses_grids_that_pd_step_would_step_differently(Grid, setting):
    """A second-order outer integrator or an edge refresh changes what pd_step
    computes; the fixed-scratch call runs neither, so it refuses such a grid
    instead of silently taking forward-Euler steps with fixed edge data."""
    from paper_2405_08764_gb300 import _native as N
    p = CASES["c1_m7"]
    if setting == "q_refresh":
        g = Grid(dict(p, q_refresh=2), prec="fp64", persistent=False)
    else:
        g = Grid(p, prec="fp64", persistent=False, integrator=setting)
    U = g.init_field()
    before = U.clone()
    with pytest.raises(N.PDError) as e:
        g.step_noalloc(U, 0.0, 0.0, 2)
    assert e.value.status == N.PD_EINVAL
    g.sync()
    assert torch.equal(U, before)
