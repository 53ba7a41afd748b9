"""Second-order projective integrators of pd_step (Heun, AB2) against the
oracle of oracle/integrators.py: FP64 within 1e-12 and FP32 within 1e-4
relative L2, on problems with a time-dependent source and Dirichlet data, a
heterogeneous tensor with a seeded source, and a periodic annulus; plus the
accuracy gain at equal macro step on the manufactured solution."""
import numpy as np
import pytest

from oracle import integrators as R
from paper_2405_08764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "c1": W.c1_manufactured(n=10, m=7),
    "c2s": W.c2_heterogeneous(n=14, m=11, n_macro=6),
    "c3s": W.c3_annulus(n_r=11, n_theta=24, m=9),
    "m5_macro": dict(W.c1_manufactured(n=9, m=5), restrict="macro"),
}


@pytest.fixture(scope="module")
def Grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_08764_gb300.api import Grid
    return Grid


@pytest.mark.parametrize("kind", ["heun", "ab2"])
@pytest.mark.parametrize("name", list(CASES))
def test_matches_oracle(Grid, orc, name, kind):
    p = CASES[name]
    o = orc.Oracle(p)
    dtm = 0.4 * o.dt_macro()
    n = 5
    step = R.step_heun if kind == "heun" else R.step_ab2
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        g = Grid(p, prec=prec, integrator=kind)
        U = g.init_field()
        U0 = U.cpu().numpy()
        g.step(U, 0.1, dtm, n)
        g.sync()
        want = step(o, U0, 0.1, dtm, n)
        err = np.linalg.norm(U.cpu().numpy() - want) / np.linalg.norm(want)
        assert err <= tol, (name, kind, prec, err)


def test_second_order_is_more_accurate_at_the_same_step(Grid, orc):
    """Manufactured solution, macro steps near the explicit bound: against a
    fine-step Heun run on the same grid, Heun and AB2 leave a much smaller
    time error than forward Euler."""
    p = W.c1_manufactured(n=8, m=5)
    o = orc.Oracle(p)
    T = 8 * 0.9 * o.dt_macro()
    errs = {}
    ref = None
    for kind, n in (("heun", 256), ("euler", 8), ("heun", 8), ("ab2", 8)):
        g = Grid(p, prec="fp64", integrator=kind)
        U = g.init_field()
        g.step(U, 0.0, T / n, n)
        g.sync()
        if ref is None:
            ref = U.clone()
            continue
        errs[kind] = (torch.linalg.norm(U - ref) / torch.linalg.norm(ref)).item()
    assert errs["heun"] < 0.2 * errs["euler"] and errs["ab2"] < 0.3 * errs["euler"], errs
    print("time error at 8 steps: euler %.2e heun %.2e ab2 %.2e" % (errs["euler"], errs["heun"], errs["ab2"]))


def test_unsupported_grids_are_refused(Grid):
    from paper_2405_08764_gb300 import _native as N
    g = Grid([CASES["c1"], CASES["c1"]], prec="fp32", integrator="heun")
    U = g.init_field()
    with pytest.raises(N.PDError) as e:
        g.step(U, 0.0, 1e-3, 1)
    assert e.value.status == N.PD_EINVAL
