"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Tolerances: all-FP64 path within relative L2 1e-12 of the
oracle at final time; FP32 bursts within 1e-4; integer layout (patch and node
indexing) exact."""
import math

import numpy as np
import pytest

from paper_2405_08764_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cases():
    c2s = W.c2_heterogeneous(n=16, m=11, n_macro=12)
    c3s = W.c3_annulus(n_r=11, n_theta=25, m=9)
    p411 = W.paper_cdr(False, lam=0.1, n=10, m=11)
    p412 = W.paper_cdr(True, lam=0.2, n=9, m=7)
    macro = dict(W.c1_manufactured(n=9, m=5, n_macro=6), restrict="macro")
    m3 = W.base(n_xi=7, n_eta=5, m_xi=3, m_eta=3, k_micro=1, M=(0.7, 0.1, 1.1), va=(0.5, 0, 0),
                vb=(-0.4, 0, 0), f0=0.3, src="mms_sinprod", time="exp", tc=-1.0, sol="sinprod_decay",
                init="exact", n_macro=5)
    tiny = W.base(n_xi=2, n_eta=2, m_xi=9, m_eta=9, init="bump", n_macro=3)
    polar_aniso = W.base(n_xi=13, n_eta=6, periodic_xi=1, box=(0, 2 * math.pi, 0, 1), map="polar",
                         map_p=(0.8, 2.2, 1.0, 0), m_xi=7, m_eta=7, M=(1.0, 0.2, 0.5),
                         va=(0.3, 0.0, 0.0), vb=(0.0, 0.0, 0.2), f0=0.4, init="bump", n_macro=6,
                         four=dict(c=[0.05, -0.03, 0.02], phi=[0.2, 1.0, 2.0], ra=0.8, rb=2.2))
    c1 = W.c1_manufactured()
    return {"c1": c1, "c2s": c2s, "c3s": c3s, "p411": p411, "p412": p412, "macro": macro, "m3": m3,
            "tiny": tiny, "polar_aniso": polar_aniso}


CASES = _cases()


@pytest.fixture(scope="module")
def env(orc):
    from paper_2405_08764_gb300.api import Grid
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return Grid


def _steps(p, o):
    dtm = p["dt_macro"] if p.get("dt_macro") else 0.5 * o.dt_macro()
    n = p.get("n_macro", 5)
    if n > 50:
        n = 50
    return dtm, n


@pytest.mark.parametrize("name", list(CASES))
def test_coefficients_match_oracle(env, orc, name):
    p = CASES[name]
    o = orc.Oracle(p)
    g = env(p, prec="fp64")
    got = g.coeffs().cpu().numpy().reshape(-1, 8)
    xi, eta = o.micro_coords()
    want = np.array([o.coeffs(a, b) for a, b in zip(xi, eta)])
    if p["src"] == "gauss_patch":
        want[:, 6] *= np.repeat(p["src_amp"], o.mx * o.my)
    # identically-zero channels (beta on orthogonal maps with isotropic K) are
    # compared on the scale of the diffusion coefficients
    floor = np.abs(want[:, [0, 2]]).max()
    for k in range(7):
        scale = max(np.abs(want[:, k]).max(), floor if k < 6 else 1e-300)
        assert np.abs(got[:, k] - want[:, k]).max() <= 1e-13 * scale, (name, k)


@pytest.mark.parametrize("name", list(CASES))
def test_step_sizes_match_oracle(env, orc, name):
    p = CASES[name]
    o = orc.Oracle(p)
    i = env(p, prec="fp64").info()
    assert i["n_patch"] == o.n_patch and i["n_macro"] == o.n_macro
    np.testing.assert_allclose(i["dt_micro"], o.dt_micro(), rtol=1e-12)
    np.testing.assert_allclose(i["dt_macro_suggested"], o.dt_macro(), rtol=1e-12)
    np.testing.assert_allclose(i["tau"], p["k_micro"] * o.dt_micro(), rtol=1e-12)


@pytest.mark.parametrize("name", ["c1", "c3s", "p411", "tiny", "polar_aniso"])
def test_initial_field_matches_oracle(env, orc, name):
    p = CASES[name]
    o = orc.Oracle(p)
    g = env(p, prec="fp64")
    for t in (0.0, 0.013):
        got = g.init_field(t=t).cpu().numpy()
        want = o.init_field(t=t)
        assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1e-300), name
    pa = W.paper_annulus()
    g2 = env(pa, prec="fp64")
    np.testing.assert_allclose(g2.init_field().cpu().numpy(), orc.Oracle(pa).init_field(), rtol=0, atol=1e-14)


def _rand_state(o, p, seed=11):
    rng = np.random.default_rng(seed)
    U = o.apply_bc(o.init_field() + 0.05 * rng.normal(size=o.n_macro), 0.21)
    return U


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_lift_matches_oracle(env, orc, name, prec):
    p = CASES[name]
    o = orc.Oracle(p)
    g = env(p, prec=prec)
    U = _rand_state(o, p)
    Ud = torch.tensor(U, device="cuda")
    st = g.new_state()
    g.lift(Ud, 0.21, st)
    v = g.state_views(st)
    u0, edge = o.lift(U)
    r0 = o.forcing(U, 0.21)
    np.testing.assert_allclose(v["u0"].cpu().numpy(), u0, rtol=0, atol=1e-13 * np.abs(u0).max())
    me = edge.shape[2]
    np.testing.assert_allclose(v["edge"].cpu().numpy()[:, :, :me], edge, rtol=0, atol=1e-11 * max(np.abs(edge).max(), 1))
    r = v["r"].cpu().numpy().astype(np.float64)
    # the oracle applies the difference stencil to FP64 lifted values: its own
    # rounding error is bounded by ~8 eps max|u0| times the stencil weight sum,
    # and the weight sum is the micro rate bound cfl / dt
    dt = g.info()["dt_micro"]
    oracle_noise = 8 * np.finfo(float).eps * np.abs(u0).max() * p["cfl_micro"] / dt
    tol = 1e-12 if prec == "fp64" else 2e-5
    err = np.abs(r - r0).max()
    assert err <= tol * np.abs(r0).max() + oracle_noise, (name, err / np.abs(r0).max(), oracle_noise)
    assert np.all(v["w"].cpu().numpy() == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_burst_and_restrict_match_oracle(env, orc, name, prec):
    p = CASES[name]
    o = orc.Oracle(p)
    g = env(p, prec=prec)
    U = _rand_state(o, p)
    Ud = torch.tensor(U, device="cuda")
    K = p["k_micro"]
    dt = g.info()["dt_micro"]
    st = g.new_state()
    g.lift(Ud, 0.21, st)
    k1 = K // 2
    g.micro_burst(st, 0.21, k1)
    g.micro_burst(st, 0.21 + k1 * dt, K - k1)
    w = g.state_views(st)["w"].cpu().numpy().astype(np.float64)
    want = o.burst(U, 0.21, K, dt, "split")
    scale = np.abs(want).max()
    tol = 1e-9 if prec == "fp64" else 2e-5
    assert np.abs(w - want).max() <= tol * scale, (name, np.abs(w - want).max() / scale)
    dU = g.restrict(st).cpu().numpy()
    dwant = o.restrict(U, want, "split")
    assert np.abs(dU - dwant).max() <= tol * max(np.abs(dwant).max(), 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_separate_passes_on_a_grid_of_two_instances(env, orc, prec):
    """pd_lift, pd_micro_burst, pd_restrict and pd_project on a two-instance grid
    whose second instance's micro points start 81 points in, off a 16-byte
    boundary (the restriction stages such a block with plain loads, the first
    instance's 81 points through its 16-byte copies and a one-point tail): each
    instance matches the oracle to the one-instance tolerances."""
    pa, pb = CASES["tiny"], CASES["p412"]
    oa, ob = orc.Oracle(pa), orc.Oracle(pb)
    g = env([pa, pb], prec=prec)
    ia, ib = g.info(0), g.info(1)
    assert ib["point_offset"] == oa.n_patch * oa.mx * oa.my and ib["point_offset"] % 4 != 0
    Ua, Ub = _rand_state(oa, pa), _rand_state(ob, pb)
    U = np.zeros(g.n_macro_total)
    U[ia["u_offset"]:ia["u_offset"] + oa.n_macro] = Ua
    U[ib["u_offset"]:ib["u_offset"] + ob.n_macro] = Ub
    Ud = torch.tensor(U, device="cuda")
    st = g.new_state()
    g.lift(Ud, 0.21, st)
    K = min(pa["k_micro"], pb["k_micro"])
    g.micro_burst(st, 0.21, K)
    dU = g.restrict(st).cpu().numpy()
    tol = 1e-9 if prec == "fp64" else 2e-5
    dwant = []
    for k, (o, Uk, info) in enumerate(((oa, Ua, ia), (ob, Ub, ib))):
        v = g.state_views(st, k)
        u0, _ = o.lift(Uk)
        np.testing.assert_allclose(v["u0"].cpu().numpy().reshape(u0.shape), u0, rtol=0,
                                   atol=1e-13 * np.abs(u0).max())
        want = o.burst(Uk, 0.21, K, info["dt_micro"], "split")
        w = v["w"].cpu().numpy().astype(np.float64)
        assert np.abs(w - want).max() <= tol * np.abs(want).max(), (k, prec)
        dk = o.restrict(Uk, want, "split")
        po = info["patch_offset"]
        got = dU[po:po + o.n_patch]
        assert np.abs(got - dk).max() <= tol * max(np.abs(dk).max(), 1e-300), (k, prec)
        dwant.append((o, Uk, info, dk))
    dUd = torch.tensor(dU, device="cuda")
    g.project(Ud, dUd, 0.3, 0.01)
    Uo = Ud.cpu().numpy()
    for o, Uk, info, _ in dwant:
        po, uo = info["patch_offset"], info["u_offset"]
        want = o.project(Uk, dU[po:po + o.n_patch], 0.3, 0.01, info["tau"])
        np.testing.assert_allclose(Uo[uo:uo + o.n_macro], want, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("name", ["c1", "p411", "c3s", "polar_aniso"])
def test_project_matches_oracle(env, orc, name):
    p = CASES[name]
    o = orc.Oracle(p)
    g = env(p, prec="fp64")
    rng = np.random.default_rng(5)
    U = _rand_state(o, p)
    dU = rng.normal(size=o.n_patch) * 1e-3
    Ud = torch.tensor(U, device="cuda")
    g.project(Ud, torch.tensor(dU, device="cuda"), 0.3, 0.01)
    want = o.project(U, dU, 0.3, 0.01, g.info()["tau"])
    np.testing.assert_allclose(Ud.cpu().numpy(), want, rtol=1e-14, atol=1e-15)


def _run_both(env, orc, p, prec, n=None, graphs=True):
    o = orc.Oracle(p)
    dtm, nn = _steps(p, o)
    n = nn if n is None else n
    g = env(p, prec=prec, graphs=graphs)
    U = g.init_field()
    U0 = U.cpu().numpy()
    g.step(U, p.get("t0", 0.0), dtm, n)
    g.sync()
    want = o.step(U0, p.get("t0", 0.0), dtm, n)
    return U.cpu().numpy(), want, g


@pytest.mark.parametrize("name", list(CASES))
def test_step_fp64_within_1e12_of_oracle(env, orc, name):
    got, want, _ = _run_both(env, orc, CASES[name], "fp64")
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-12, (name, err)


@pytest.mark.parametrize("name", list(CASES))
def test_step_fp32_within_1e4_of_oracle(env, orc, name):
    got, want, _ = _run_both(env, orc, CASES[name], "fp32")
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-4, (name, err)


def test_c1_full_run_fp64_and_fp32(env, orc):
    """Configuration 1 as specified: 50 macro steps to t = 0.5."""
    p = W.c1_manufactured()
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        got, want, _ = _run_both(env, orc, p, prec, n=50)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= tol, prec


def test_graph_replay_equals_direct_launches(env, orc):
    p = CASES["c2s"]
    a, _, g1 = _run_both(env, orc, p, "fp32", graphs=True)
    b, _, _ = _run_both(env, orc, p, "fp32", graphs=False)
    np.testing.assert_array_equal(a, b)
    # replaying the cached graph from the same start gives the same bits
    U = g1.init_field()
    dtm = 0.5 * orc.Oracle(p).dt_macro()
    n = _steps(p, orc.Oracle(p))[1]
    g1.step(U, 0.0, dtm, n)
    g1.step(U, n * dtm, dtm, n)
    g1.sync()
    U2 = g1.init_field()
    g1.step(U2, 0.0, dtm, 2 * n)
    g1.sync()
    np.testing.assert_allclose(U.cpu().numpy(), U2.cpu().numpy(), rtol=0, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_separate_passes_compose_to_the_fused_step(env, orc, prec):
    p = CASES["c2s"]
    o = orc.Oracle(p)
    g = env(p, prec=prec)
    dtm = 0.5 * o.dt_macro()
    U1 = g.init_field()
    U1 += 0.01 * torch.rand_like(U1)
    U2 = U1.clone()
    g.step(U1, 0.05, dtm, 1)
    st = g.new_state()
    g.lift(U2, 0.05, st)
    g.micro_burst(st, 0.05, p["k_micro"])
    dU = g.restrict(st)
    U0 = U2.clone()
    g.project(U2, dU, 0.05, dtm)
    g.sync()
    a, b, u0 = U1.cpu().numpy(), U2.cpu().numpy(), U0.cpu().numpy()
    # compare the macro increments: same arithmetic, possibly different FP32
    # contraction between the fused and the separate kernels
    tol = 1e-13 if prec == "fp64" else 1e-5
    inc = np.abs(a - u0).max()
    assert np.abs(a - b).max() <= tol * inc, (np.abs(a - b).max(), inc)


@pytest.mark.parametrize("mx,my", [(13, 13), (7, 9), (11, 5)])
def test_generic_path_for_other_micro_sizes(env, orc, mx, my):
    p = W.c2_heterogeneous(n=8, m=mx, n_macro=3)
    p["m_eta"] = my
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        got, want, _ = _run_both(env, orc, p, prec)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= tol, (mx, my, prec)


def test_full_size_heterogeneous_workload_fp32(env, orc):
    """The 65 x 65, m = 11, 200-step workload in the launch configuration the
    benchmark times, against the oracle's full run."""
    p = W.c2_heterogeneous()
    got, want, g = _run_both(env, orc, p, "fp32", n=200)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-4, err


def test_full_size_heterogeneous_workload_fp64(env, orc):
    """The same full run in FP64 (per-step and persistent kernels alike run
    the FP64 bursts) within the FP64 bound of the oracle."""
    p = W.c2_heterogeneous()
    got, want, g = _run_both(env, orc, p, "fp64", n=200)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 1e-12, err


def _literal_tol(o, p, dtm, n):
    """FP64 bound against the literal recursion: the parity bound 1e-12 plus the
    literal form's own cancellation.  The literal burst evolves u itself, so each
    of its K forward-Euler updates rounds at |u| eps, and the restricted change
    U1 - U0 that the step divides by tau keeps that absolute error; the macro
    step multiplies it by dt_macro / tau.  Over n macro steps: n K (dt/tau) eps,
    relative to |U| (a worst case: the roundings are not all aligned)."""
    return 1e-12 + n * p["k_micro"] * (dtm / o.tau()) * 2.0 ** -52


@pytest.mark.parametrize("name", ["c1", "c2s", "p411", "p412", "macro", "polar_aniso", "m3", "tiny"])
def test_step_fp64_against_the_literal_recursion(env, orc, name):
    """The GPU evaluates each burst in the split form (departure from the lift,
    closed-form forcing); the oracle's literal form runs eq. (Computational_Problem)
    on u itself with the explicit ghost points of the edge data, restricts u and
    forms (U1 - U0)/tau as eq. (Time_Derivative) prints it.  The two meet within
    the FP64 bound widened by the literal form's cancellation."""
    p = CASES[name]
    o = orc.Oracle(p)
    dtm, n = _steps(p, o)
    g = env(p, prec="fp64")
    U = g.init_field()
    U0 = U.cpu().numpy()
    g.step(U, p.get("t0", 0.0), dtm, n)
    g.sync()
    want = o.step(U0, p.get("t0", 0.0), dtm, n, form="literal")
    err = np.linalg.norm(U.cpu().numpy() - want) / np.linalg.norm(want)
    assert err <= _literal_tol(o, p, dtm, n), (name, err, _literal_tol(o, p, dtm, n))


def test_full_size_heterogeneous_workload_against_the_literal_recursion(env, orc):
    """65 x 65, m = 11, 200 macro steps in FP64 against the oracle's literal
    recursion (tau ~ dt_macro / 60 here, the regime where the literal quotient
    cancels most)."""
    p = W.c2_heterogeneous()
    o = orc.Oracle(p)
    dtm, _ = _steps(p, o)
    g = env(p, prec="fp64")
    U = g.init_field()
    U0 = U.cpu().numpy()
    g.step(U, 0.0, dtm, 200)
    g.sync()
    want = o.step(U0, 0.0, dtm, 200, form="literal")
    err = np.linalg.norm(U.cpu().numpy() - want) / np.linalg.norm(want)
    assert err <= _literal_tol(o, p, dtm, 200), err


def test_batched_instances_against_the_literal_recursion(env, orc):
    """Six uneven batched instances (work-queue kernel, metric tables) in FP64
    against the literal recursion, each at its own suggested macro step."""
    probs = [dict(W.c4_instance(i), n_xi=min(W.c4_instance(i)["n_xi"], 32),
                  n_eta=min(W.c4_instance(i)["n_eta"], 32)) for i in range(6)]
    g = env(probs, prec="fp64")
    U = g.init_field()
    U0 = U.cpu().numpy()
    g.step(U, 0.0, 0.0, 6)
    g.sync()
    got = U.cpu().numpy()
    for k, p in enumerate(probs):
        i = g.info(k)
        a, nn = i["u_offset"], i["n_macro"]
        o = orc.Oracle(p)
        want = o.step(U0[a:a + nn], 0.0, o.dt_macro(), 6, form="literal")
        err = np.linalg.norm(got[a:a + nn] - want) / np.linalg.norm(want)
        assert err <= _literal_tol(o, p, o.dt_macro(), 6), (k, p["map"], p["m_xi"], err)


@pytest.mark.parametrize("field", ["burst", "mixed_signs"])
def test_fp32_restriction_sum_error_is_bounded(env, field):
    """The FP32 path sums the trapezoid average of the departure in FP32 (the
    separate pass: four strided FMA chains and a two-level shuffle tree; the
    fused kernels: column sums and a log2(m)-level tree), then forms dU in FP64.
    Against the exact sum of the same FP32 values, the error of any summation
    order with at most n additions on a path is bounded by
    gamma_n * sum |weight * w| (gamma_n = n u / (1 - n u), u = 2^-24), and the
    restricted change must stay within it for the departures of a real burst
    and for a field of random signs."""
    p = CASES["c2s"]
    g = env(p, prec="fp32")
    i = g.info()
    mx, my = i["m_xi"], i["m_eta"]
    U = g.init_field()
    st = g.new_state()
    g.lift(U, 0.0, st)
    g.micro_burst(st, 0.0, p["k_micro"])
    v = g.state_views(st)
    if field == "mixed_signs":
        rng = np.random.default_rng(7)
        v["w"].copy_(torch.tensor(rng.normal(size=tuple(v["w"].shape)) * 1e-6, dtype=torch.float32))
    dU = g.restrict(st).cpu().numpy()
    w = v["w"].cpu().numpy().astype(np.float64)
    bias = v["bias"].cpu().numpy()
    tw = np.outer(np.where((np.arange(my) == 0) | (np.arange(my) == my - 1), 0.5, 1.0),
                  np.where((np.arange(mx) == 0) | (np.arange(mx) == mx - 1), 0.5, 1.0))
    inv_nn = 1.0 / ((mx - 1) * (my - 1))
    exact = (w * tw).sum(axis=(1, 2)) * inv_nn + bias
    mag = (np.abs(w) * tw).sum(axis=(1, 2)) * inv_nn
    n_add = max(-(-mx * my // 4) + 2, mx + int(np.ceil(np.log2(mx)))) + 1
    u = 2.0 ** -24
    gamma = n_add * u / (1 - n_add * u)
    assert np.all(np.abs(dU - exact) <= gamma * mag + 1e-300), np.max(np.abs(dU - exact) / (gamma * mag))
    if field == "burst":
        # departures of one sign inside a patch: the sum's relative error is far
        # below the 1e-4 bound of the FP32 path
        assert np.max(np.abs(dU - exact) / np.maximum(np.abs(exact - bias), 1e-300)) <= 1e-5


def test_full_size_annulus_sampled_patches(env, orc):
    """128 x 512 annulus (m = 9): one macro step of dU on the GPU against the
    oracle on 300 sampled patches (including the periodic seam and both walls)."""
    p = W.c3_annulus()
    o = orc.Oracle(p)
    g = env(p, prec="fp32")
    U = g.init_field()
    st = g.new_state()
    g.lift(U, 0.0, st)
    g.micro_burst(st, 0.0, p["k_micro"])
    dU = g.restrict(st).cpu().numpy()
    rng = np.random.default_rng(0)
    ncol = p["n_xi"]
    sel = np.unique(np.concatenate([rng.integers(0, o.n_patch, 280), [0, ncol - 1, ncol, o.n_patch - 1,
                                                                        o.n_patch - ncol]]))
    want = o.patch_dU(U.cpu().numpy(), 0.0, sel)
    scale = np.abs(want).max()
    assert np.abs(dU[sel] - want).max() <= 2e-5 * scale


def test_nonfinite_values_are_reported(env, orc):
    from paper_2405_08764_gb300 import _native as N
    p = W.c1_manufactured(n=8)
    g = env(p, prec="fp32")
    U = g.init_field()
    g.step(U, 0.0, 1e6, 40)   # far above the macro stability bound
    with pytest.raises(N.PDError) as e:
        g.sync()
    assert e.value.status == N.PD_ENUMERIC


def test_checkpoint_roundtrip(env, orc, tmp_path):
    p = CASES["c3s"]
    g = env(p, prec="fp32")
    U = g.init_field()
    g.step(U, 0.0, 1e-5, 3)
    path = str(tmp_path / "ck.bin")
    g.save_checkpoint(U, 3e-5, 3, path)
    V = torch.zeros_like(U)
    t, s = g.load_checkpoint(V, path)
    assert t == 3e-5 and s == 3
    assert torch.equal(U, V)
    g2 = env(CASES["c2s"], prec="fp32")
    from paper_2405_08764_gb300 import _native as N
    with pytest.raises(N.PDError):
        g2.load_checkpoint(torch.zeros(g2.n_macro_total, dtype=torch.float64, device="cuda"), path)


@pytest.mark.parametrize("name", ["c3s", "polar_aniso", "batch"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resume_from_checkpoint_equals_uninterrupted_run(env, tmp_path, name, prec):
    """n macro steps, a checkpoint, a fresh grid that loads it and m more steps
    give bitwise the field of n + m uninterrupted steps.  The problems carry no
    time-dependent source or boundary data, so both runs see the same time
    levels exactly (with time dependence the resumed time origin t0 + n dt is
    rounded once more).  Covers the persistent dataflow path (annulus), the
    per-step fused path with a cross term (anisotropic annulus) and the batched
    work queue (six uneven instances)."""
    probs = [dict(W.c4_instance(i), n_xi=min(W.c4_instance(i)["n_xi"], 32),
                  n_eta=min(W.c4_instance(i)["n_eta"], 32)) for i in range(6)] if name == "batch" else CASES[name]
    n, m = 5, 4
    dtm = 0.0 if name == "batch" else 0.5 * env(probs, prec="fp64").info()["dt_macro_suggested"]
    ref = env(probs, prec=prec)
    U = ref.init_field()
    ref.step(U, 0.0, dtm, n + m)
    ref.sync()
    a = env(probs, prec=prec)
    V = a.init_field()
    a.step(V, 0.0, dtm, n)
    path = str(tmp_path / "resume.bin")
    a.save_checkpoint(V, n * dtm, n, path)
    del a
    b = env(probs, prec=prec)
    W2 = torch.full_like(V, float("nan"))
    t, s = b.load_checkpoint(W2, path)
    assert s == n and t == n * dtm
    b.step(W2, t, dtm, m)
    b.sync()
    assert torch.equal(W2, U), float((W2 - U).abs().max())


def test_invalid_calls_are_rejected(env, orc):
    from paper_2405_08764_gb300 import _native as N
    g = env(CASES["c1"], prec="fp32")
    st = g.new_state()
    with pytest.raises(N.PDError):
        g.micro_burst(st, 0.0, 5000)
    with pytest.raises(N.PDError):
        g.project(g.new_field(), torch.zeros(g.n_patch_total, dtype=torch.float64, device="cuda"), 0.0, -1.0)
    U = g.new_field()
    with pytest.raises(N.PDError):
        g.lift(U, 0.0, st[1:])   # misaligned state buffer


def test_largest_micro_patch_and_longest_burst(env, orc):
    """The size limits of the descriptors: m = 32 (generic shared-memory
    burst) and K = 4096 micro steps per burst, FP64 and FP32."""
    big_m = W.base(n_xi=4, n_eta=3, m_xi=32, m_eta=32, k_micro=20, M=(0.7, 0.1, 1.1), va=(0.5, 0, 0),
                   vb=(-0.4, 0, 0), f0=0.3, init="bump", n_macro=2)
    long_k = W.base(n_xi=4, n_eta=4, m_xi=3, m_eta=3, k_micro=4096, cfl_micro=0.01, M=(0.7, 0.1, 1.1),
                    va=(0.5, 0, 0), vb=(-0.4, 0, 0), f0=0.3, init="bump", n_macro=2)
    for p in (big_m, long_k):
        for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
            got, want, _ = _run_both(env, orc, p, prec)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= tol, (p["m_xi"], p["k_micro"], prec)


def test_zero_steps_and_empty_bursts_leave_the_state_alone(env, orc):
    p = CASES["c2s"]
    g = env(p, prec="fp32")
    U = g.init_field()
    U0 = U.clone()
    g.step(U, 0.0, 1e-5, 0)
    g.sync()
    assert torch.equal(U, U0)
    st = g.new_state()
    g.lift(U, 0.0, st)
    before = st.clone()
    g.micro_burst(st, 0.0, 0)
    g.sync()
    assert torch.equal(st, before)
