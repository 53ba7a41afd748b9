"""Batched execution of many uneven instances (work-queue kernel) and the
table coefficient mode, against the CPU oracle instance by instance."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _c4_subset(n, cap=32, seed0=4):
    out = []
    for i in range(n):
        p = W.c4_instance(i, seed0)
        p["n_xi"] = min(p["n_xi"], cap)
        p["n_eta"] = min(p["n_eta"], cap)
        out.append(p)
    return out


@pytest.fixture(scope="module")
def Grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_08764_gb300.api import Grid
    return Grid


def _split(g, U):
    out = []
    for k in range(len(g.probs)):
        i = g.info(k)
        out.append(U[i["u_offset"]:i["u_offset"] + i["n_macro"]].cpu().numpy())
    return out


def _oracle_runs(orc, probs, n):
    res = []
    for p in probs:
        o = orc.Oracle(p)
        dtm = o.dt_macro()          # pd_step(dt_macro <= 0) uses each instance's suggested step
        res.append(o.step(o.init_field(), 0.0, dtm, n))
    return res


def test_table_coefficients_match_oracle(Grid, orc):
    probs = _c4_subset(12)
    g = Grid(probs, prec="fp64")
    for k, p in enumerate(probs):
        assert g.info(k)["exec_path"] == 3
        o = orc.Oracle(p)
        got = g.coeffs(k).cpu().numpy().reshape(-1, 8)[:, :6]
        xi, eta = o.micro_coords()
        want = np.array([o.coeffs(a, b)[:6] for a, b in zip(xi, eta)])
        floor = np.abs(want[:, [0, 2]]).max()
        # the table form (1/X', X''/X'^3) and the general metric formula are two FP64
        # arrangements of the same closed form; near a tanh-clustered edge X' ~ 5e-3
        # and their rounding differs by ~1e-13 relative
        for c in range(6):
            scale = max(np.abs(want[:, c]).max(), floor)
            assert np.abs(got[:, c] - want[:, c]).max() <= 1e-12 * scale, (k, p["map"], c)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_batched_uneven_instances_match_oracle(Grid, orc, prec, tol):
    probs = _c4_subset(24)
    g = Grid(probs, prec=prec)
    U = g.init_field()
    g.step(U, 0.0, 0.0, 8)        # each instance at half its explicit macro bound
    g.sync()
    got = _split(g, U)
    want = _oracle_runs(orc, probs, 8)
    for k, (a, b) in enumerate(zip(got, want)):
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= tol, (k, probs[k]["map"], probs[k]["m_xi"], err)


def test_batched_equals_single_instance_grids_bitwise(Grid):
    probs = _c4_subset(10)
    g = Grid(probs, prec="fp64")
    U = g.init_field()
    g.step(U, 0.0, 0.0, 5)
    g.sync()
    got = _split(g, U)
    for k, p in enumerate(probs):
        s = Grid(p, prec="fp64", storage="tables", autotune=False)
        V = s.init_field()
        s.step(V, 0.0, 0.0, 5)
        s.sync()
        np.testing.assert_array_equal(got[k], V.cpu().numpy())


def test_table_and_record_storage_agree(Grid):
    probs = _c4_subset(6)
    a = Grid(probs, prec="fp64", storage="tables")
    b = Grid(probs, prec="fp64", storage="records")
    Ua, Ub = a.init_field(), b.init_field()
    a.step(Ua, 0.0, 0.0, 6)
    b.step(Ub, 0.0, 0.0, 6)
    a.sync(), b.sync()
    x, y = Ua.cpu().numpy(), Ub.cpu().numpy()
    assert np.abs(x - y).max() <= 1e-12 * np.abs(y).max()


def test_mixed_problems_with_sources_and_dirichlet_data(Grid, orc):
    """Records storage in one batch: manufactured source (time factor exp(-t)),
    exponential Dirichlet data, tensor diffusion with a per-patch amplitude
    source (time factor sin), a periodic annulus; different micro sizes."""
    probs = [W.c1_manufactured(n=8, m=7), W.paper_cdr(True, lam=0.2, n=9, m=9),
             W.c2_heterogeneous(n=12, m=11), W.c3_annulus(n_r=9, n_theta=14, m=5)]
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        g = Grid(probs, prec=prec)
        U = g.init_field()
        g.step(U, 0.0, 0.0, 6)
        g.sync()
        got = _split(g, U)
        want = _oracle_runs(orc, probs, 6)
        for k, (a, b) in enumerate(zip(got, want)):
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert err <= tol, (prec, k, err)


def test_separate_passes_with_mixed_micro_sizes(Grid, orc):
    probs = _c4_subset(5)
    g = Grid(probs, prec="fp64")
    U = g.init_field()
    rng = np.random.default_rng(2)
    U += torch.tensor(0.01 * rng.normal(size=U.numel()), device="cuda")
    st = g.new_state()
    g.lift(U, 0.0, st)
    g.micro_burst(st, 0.0, probs[0]["k_micro"])      # every instance has K = 20
    dU = g.restrict(st).cpu().numpy()
    Uh = _split(g, U)
    for k, p in enumerate(probs):
        o = orc.Oracle(p)
        dt = g.info(k)["dt_micro"]
        w = o.burst(Uh[k], 0.0, p["k_micro"], dt, "split")
        want = o.restrict(Uh[k], w, "split")
        i = g.info(k)
        mine = dU[i["patch_offset"]:i["patch_offset"] + i["n_patch"]]
        assert np.abs(mine - want).max() <= 1e-10 * max(np.abs(want).max(), 1e-300), k
        v = g.state_views(st, k)
        u0, _ = o.lift(Uh[k])
        np.testing.assert_allclose(v["u0"].cpu().numpy(), u0, rtol=0, atol=1e-13 * np.abs(u0).max())


def test_autotuner_picks_a_configuration_and_keeps_results(Grid):
    probs = _c4_subset(8)
    g = Grid(probs, prec="fp32", autotune=False)
    U = g.init_field()
    g.step(U, 0.0, 0.0, 4)
    g.sync()
    block, half = g.autotune(2)
    assert block in (64, 128, 256)
    V = g.init_field()
    g.step(V, 0.0, 0.0, 4)
    g.sync()
    np.testing.assert_array_equal(U.cpu().numpy(), V.cpu().numpy())


def test_batch_with_a_single_patch_instance(Grid, orc):
    """A 2 x 2 macro grid has one patch: one partial patch group and a
    boundary chunk of eight nodes in the same queue as larger instances."""
    probs = [W.base(n_xi=2, n_eta=2, m_xi=7, m_eta=7, init="bump"), _c4_subset(3)[2], _c4_subset(3)[0]]
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        g = Grid(probs, prec=prec)
        U = g.init_field()
        g.step(U, 0.0, 0.0, 4)
        g.sync()
        got = _split(g, U)
        want = _oracle_runs(orc, probs, 4)
        for k, (a, b) in enumerate(zip(got, want)):
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
            assert err <= tol, (prec, k, err)


def test_full_size_batch_sampled_instances(Grid, orc):
    """The 4096-instance batch (N up to 128, m up to 11) in the launch
    configuration the benchmark times (FP32, autotuned work queue, each
    instance at its own suggested macro step), three macro steps, against the
    oracle on sampled instances: the largest ones, every map and micro size,
    both ends of the queue."""
    probs = W.c4_batch(4096)
    g = Grid(probs, prec="fp32")
    U = g.init_field()
    U0 = U.cpu().numpy()
    g.step(U, 0.0, 0.0, 3)
    g.sync()
    got = U.cpu().numpy()
    sel = {0, len(probs) - 1}
    sel |= set([k for k, p in enumerate(probs) if p["n_xi"] == 128 and p["m_xi"] == 11][:2])
    for key, vals in (("map", ("identity", "tanh", "polar")), ("m_xi", (5, 7, 9, 11))):
        for v in vals:
            sel.add(next(k for k, p in enumerate(probs) if p[key] == v and p["n_xi"] >= 64))
    for k in sorted(sel):
        i = g.info(k)
        o = orc.Oracle(probs[k])
        a = i["u_offset"]
        want = o.step(U0[a:a + i["n_macro"]], 0.0, o.dt_macro(), 3)
        err = np.linalg.norm(got[a:a + i["n_macro"]] - want) / np.linalg.norm(want)
        assert err <= 1e-4, (k, probs[k]["map"], probs[k]["n_xi"], probs[k]["m_xi"], err)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_batched_macro_reference_matches_oracle(Grid, orc, prec, tol):
    """The printed restriction reference U0 = U_ij (MACRO) on the batched path:
    the interpolant's c20, c02 enter the reference offset in FP64."""
    probs = [dict(p, restrict="macro") for p in _c4_subset(6)]
    g = Grid(probs, prec=prec)
    U = g.init_field()
    g.step(U, 0.0, 0.0, 5)
    g.sync()
    got = _split(g, U)
    want = _oracle_runs(orc, probs, 5)
    for k, (a, b) in enumerate(zip(got, want)):
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= tol, (k, probs[k]["map"], probs[k]["m_xi"], err)
