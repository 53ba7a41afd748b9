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
