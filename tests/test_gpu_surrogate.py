"""The surrogate on a grid (include/pd_surrogate.h) against the CPU oracle:
features, training targets, the check estimate F1 and the full-burst F, the
network's F, the all-fallback limit (the plain scheme) and the accept-all
limit, and end to end: a network trained on the GPU from patch-solver data
serves most patches of an unseen field within the 1e-3 tolerance of the plain
scheme, where an untrained one serves none."""
import math

import numpy as np
import pytest

from oracle import Oracle
from oracle import surrogate as S
from paper_2405_08764_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_08764_gb300 import api
    return api


def _small(seed=5):
    return W.c5_surrogate_field(n_r=15, n_theta=48, m=9, seed=seed)


def _net(api, seed=3, max_batch=256):
    net = api.MLP(max_batch)
    th = S.init_params(seed)
    p = S.unflatten(th)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.normal(size=p[k].shape)
    net.set_params(S.flatten(p).astype(np.float32))
    mu = rng.normal(size=S.N_IN).astype(np.float32) * 0.1
    sg = rng.uniform(0.5, 2.0, S.N_IN).astype(np.float32)
    net.set_norm(mu, sg, 0.01)
    return net


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_raw_features_match_oracle(api, prec):
    p = _small()
    g = api.Grid(p, prec=prec)
    s = api.Surrogate(g, _net(api))
    U = g.init_field()
    f = s.features(U, standardised=False, raw=True)
    o = Oracle(p)
    X, sc, R = S.features(o, U.cpu().numpy())
    got = f["X_raw"].cpu().numpy().astype(np.float64)
    # FP32 outputs of FP64 arithmetic done in another order
    np.testing.assert_allclose(got, X, rtol=2e-6, atol=2e-7)
    np.testing.assert_allclose(f["Rs"].cpu().numpy(), R * sc, rtol=1e-11)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_targets_and_check_estimate_match_oracle(api, prec, tol):
    p = _small()
    g = api.Grid(p, prec=prec)
    s = api.Surrogate(g, _net(api))
    U = g.init_field()
    o = Oracle(p)
    Uh = U.cpu().numpy()
    X, sc, R = S.features(o, Uh)
    FK = S.patch_F(o, Uh, 0.0)
    F1 = S.patch_F(o, Uh, 0.0, 1)
    ev = s.evaluate(U, 0.0, F_hat=False)
    np.testing.assert_allclose(ev["F"].cpu().numpy(), FK, rtol=0, atol=tol * np.abs(FK).max())
    np.testing.assert_allclose(ev["F1"].cpu().numpy(), F1, rtol=0, atol=tol * np.abs(F1).max())
    f = s.features(U, standardised=False, raw=True)
    y = s.targets(U, 0.0, f["Rs"]).cpu().numpy()
    want = FK / (R * sc)
    np.testing.assert_allclose(y, want, rtol=0, atol=max(tol, 1e-6) * np.abs(want).max())


def test_network_F_matches_oracle(api):
    p = _small()
    g = api.Grid(p, prec="fp32")
    net = _net(api)
    s = api.Surrogate(g, net)
    U = g.init_field()
    Fh = s.evaluate(U, 0.0, F1=False, F=False)["F_hat"].cpu().numpy()
    o = Oracle(p)
    X, sc, R = S.features(o, U.cpu().numpy())
    mu, sg, ys = net.norm()
    Xs = (X.astype(np.float32) - mu) / sg
    y, _ = S.forward(net.params().astype(np.float64), Xs.astype(np.float64), round_bf16=True)
    want = y * ys * R * sc
    # hidden-layer tanh approximation and BF16 rounding flips (see test_gpu_mlp._close)
    err = np.abs(Fh - want) / np.abs(want).max()
    assert np.quantile(err, 0.99) <= 2.5e-3 and err.max() <= 1e-2, (np.quantile(err, 0.99), err.max())


def test_all_fallback_is_the_plain_scheme(api):
    p = _small()
    g = api.Grid(p, prec="fp64")
    s = api.Surrogate(g, _net(api))
    U = g.init_field()
    dtm = g.info()["dt_macro_suggested"]
    s.step(U, 0.0, dtm, 4, eps=-1.0)
    g.sync()
    o = Oracle(p)
    want = o.step(o.init_field(), 0.0, dtm, 4)
    got = U.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-12
    steps, fb = s.counts()
    assert steps == fb == 4 * o.n_patch


def test_accept_all_uses_the_network(api):
    p = _small()
    g = api.Grid(p, prec="fp32")
    net = _net(api)
    s = api.Surrogate(g, net)
    U = g.init_field()
    U0 = U.clone()
    dtm = g.info()["dt_macro_suggested"]
    Fh = s.evaluate(U, 0.0, F1=False, F=False)["F_hat"]
    s.step(U, 0.0, dtm, 1, eps=float("inf"))
    g.sync()
    o = Oracle(p)
    I, J = o.patch_nodes()
    nodes = J * o.nxp + I
    d = (U - U0).cpu().numpy()[nodes]
    np.testing.assert_allclose(d, dtm * Fh.cpu().numpy(), rtol=1e-9, atol=1e-12 * np.abs(U0.cpu().numpy()).max())
    assert s.counts()[1] == 0


def _dataset(api, net, seeds, n_r, n_theta, snaps, n_noisy=4):
    """patch-solver samples from fields of the plain scheme at several times,
    each also with grid-scale perturbations of relative size 1e-9..1e-5 (the
    size the check's accepted errors leave in the field)"""
    Xs, ys = [], []
    rng = np.random.default_rng(8)
    for sd in seeds:
        p = W.c5_surrogate_field(n_r=n_r, n_theta=n_theta, m=9, seed=sd)
        g = api.Grid(p, prec="fp32")
        s = api.Surrogate(g, net)
        U = g.init_field()
        dtm = g.info()["dt_macro_suggested"]
        for k in range(snaps):
            for c in range(1 + n_noisy):
                V = U if c == 0 else s.perturb(U, 10.0 ** rng.uniform(-9, -5), int(rng.integers(1 << 62)))
                f = s.features(V, standardised=False, raw=True)
                Xs.append(f["X_raw"])
                ys.append(s.targets(V, k * 20 * dtm, f["Rs"]))
            g.step(U, k * 20 * dtm, dtm, 20)
    return torch.cat(Xs), torch.cat(ys)


def test_perturbation(api):
    p = _small()
    g = api.Grid(p, prec="fp64")
    s = api.Surrogate(g, _net(api))
    U = g.init_field()
    V = s.perturb(U, 1e-3, 77)
    o = Oracle(p)
    d = (V - U).cpu().numpy().reshape(o.nyp, o.nxp)
    assert np.all(d[0] == 0) and np.all(d[-1] == 0)
    z = d[1:-1].ravel() / (1e-3 * U.abs().max().item())
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1.0) < 0.1
    np.testing.assert_array_equal(s.perturb(U, 1e-3, 77).cpu().numpy(), V.cpu().numpy())


def test_trained_network_serves_most_patches(api):
    n_r, n_theta = 47, 192
    net = api.MLP(2048)
    Xr, yr = _dataset(api, net, range(1000, 1008), n_r, n_theta, 3)
    net.fit_norm(Xr, yr)
    X, t = net.pack(Xr, yr)
    net.init(21)
    hist = net.train(X, t, batch=2048, epochs=160, lr_max=2e-3, seed=2)
    net.sync()
    assert hist[-1] < 1e-4 * hist[0], hist[[0, -1]]

    p = W.c5_surrogate_field(n_r=n_r, n_theta=n_theta, m=9, seed=5)   # unseen field
    n_steps = 10
    plain = api.Grid(p, prec="fp32")
    Up = plain.init_field()
    dtm = plain.info()["dt_macro_suggested"]
    plain.step(Up, 0.0, dtm, n_steps)

    g = api.Grid(p, prec="fp32")
    s = api.Surrogate(g, net)
    U = g.init_field()
    s.step(U, 0.0, dtm, n_steps)
    g.sync()
    steps, fb = s.counts()
    served = 1.0 - fb / steps
    err = (torch.linalg.norm(U - Up) / torch.linalg.norm(Up)).item()
    assert err <= 1e-3, err
    print("served by the trained network: %.3f, error vs plain %.2e" % (served, err))
    assert served >= 0.5, served

    untrained = api.MLP(256)
    untrained.init(21)
    mu, sg, ys = net.norm()
    untrained.set_norm(mu, sg, ys)
    g2 = api.Grid(p, prec="fp32")
    s2 = api.Surrogate(g2, untrained)
    U2 = g2.init_field()
    s2.step(U2, 0.0, dtm, n_steps)
    g2.sync()
    st2, fb2 = s2.counts()
    assert fb2 / st2 >= 0.99


def test_full_size_annulus_sampled_patches(api):
    """The 512 x 2048-node annulus (1,044,480 patches, 9 x 9 micro, FP32) in
    the launch configuration the benchmark times: raw features, the full-burst
    F and the check estimate F1 against the oracle on sampled patches (both
    walls and the periodic seam included), the network's F_hat on those rows,
    and one surrogate macro step whose check splits the patches about evenly
    between the network and the burst fallback: at every sampled patch node
    the step adds dt F_hat where the check accepts and dt F where it falls
    back."""
    p = W.c5_surrogate_field()
    g = api.Grid(p, prec="fp32")
    net = _net(api, max_batch=4096)
    s = api.Surrogate(g, net)
    U = g.init_field()
    o = Oracle(p)
    n = o.n_patch
    ncol = p["n_xi"]
    rng = np.random.default_rng(11)
    sel = np.unique(np.concatenate([rng.integers(0, n, 250), [0, 1, ncol - 1, ncol, n - ncol, n - 1]]))
    Uh = U.cpu().numpy()

    f = s.features(U, standardised=False, raw=True)
    X, sc, R = S.features(o, Uh, sel=sel)
    np.testing.assert_allclose(f["X_raw"].cpu().numpy()[sel].astype(np.float64), X, rtol=2e-6, atol=2e-7)
    np.testing.assert_allclose(f["Rs"].cpu().numpy()[sel], R * sc, rtol=1e-11)

    ev = s.evaluate(U, 0.0)
    Fh, F1, FK = (ev[k].cpu().numpy() for k in ("F_hat", "F1", "F"))
    dt = o.dt_micro()
    wantK = o.patch_dU(Uh, 0.0, sel, dt_micro=dt) / (p["k_micro"] * dt)
    want1 = Oracle(dict(p, k_micro=1)).patch_dU(Uh, 0.0, sel, dt_micro=dt) / dt
    tol = 2e-4
    np.testing.assert_allclose(FK[sel], wantK, rtol=0, atol=tol * np.abs(wantK).max())
    np.testing.assert_allclose(F1[sel], want1, rtol=0, atol=tol * np.abs(want1).max())

    mu, sg, ys = net.norm()
    Xs = (X.astype(np.float32) - mu) / sg
    y, _ = S.forward(net.params().astype(np.float64), Xs.astype(np.float64), round_bf16=True)
    want_h = y * ys * R * sc
    err = np.abs(Fh[sel] - want_h) / np.abs(want_h).max()
    assert np.quantile(err, 0.99) <= 2.5e-3 and err.max() <= 1e-2, (np.quantile(err, 0.99), err.max())

    # the check threshold that accepts about half of the patches
    rho = math.sqrt(float(np.mean(F1 ** 2)))
    ratio = np.abs(Fh - F1) / (np.abs(F1) + rho)
    eps = float(np.median(ratio))
    U0 = U.clone()
    dtm = g.info()["dt_macro_suggested"]
    s.step(U, 0.0, dtm, 1, eps=eps)
    g.sync()
    steps, fb = s.counts()
    assert steps == n and 0.3 * n <= fb <= 0.7 * n, (steps, fb)
    I, J = o.patch_nodes()
    d = (U - U0).cpu().numpy()[J[sel] * o.nxp + I[sel]]
    r = ratio[sel]
    clear = np.abs(r - eps) > 1e-6 * eps           # decisions away from the threshold
    assert clear.sum() >= 0.9 * len(sel)
    expect = dtm * np.where(r <= eps, Fh[sel], FK[sel])
    scale = dtm * max(np.abs(Fh[sel]).max(), np.abs(FK[sel]).max())
    np.testing.assert_allclose(d[clear], expect[clear], rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_one_step_scheme_matches_oracle_with_one_micro_step(api, prec, tol):
    """pd_surrogate_step_f1 (every patch takes the check estimate F1, no network)
    is the plain scheme with bursts of one micro step: the oracle's step with
    K = 1 at the same micro step, Dirichlet data and projection."""
    p = _small()
    g = api.Grid(p, prec=prec)
    s = api.Surrogate(g, _net(api))
    dt, dtm = g.info()["dt_micro"], g.info()["dt_macro_suggested"]
    U = g.init_field()
    U0 = U.cpu().numpy()
    s.step_f1(U, 0.0, dtm, 6)
    g.sync()
    want = Oracle(dict(p, k_micro=1)).step(U0, 0.0, dtm, 6, dt)
    err = np.linalg.norm(U.cpu().numpy() - want) / np.linalg.norm(want)
    assert err <= tol, err


def test_one_step_scheme_is_within_the_check_tolerance_of_the_burst(api):
    """Section 4's tau-insensitivity on the surrogate workload: over 20 macro
    steps the scheme without the network at one micro step per burst moves the
    field by the same change as the K-step scheme to within the 1e-3 tolerance
    the surrogate is held to (1.5e-4 here), so F1 -- the estimate the residual
    check compares the network with -- is itself an admissible answer, and the
    network's gain is measured against it (bench.py --workload c5: f1_only)."""
    p = _small()
    g = api.Grid(p, prec="fp64")
    s = api.Surrogate(g, _net(api))
    dtm = g.info()["dt_macro_suggested"]
    U0 = g.init_field()
    A, B = U0.clone(), U0.clone()
    g.step(A, 0.0, dtm, 20)
    s.step_f1(B, 0.0, dtm, 20)
    g.sync()
    a, b, u0 = A.cpu().numpy(), B.cpu().numpy(), U0.cpu().numpy()
    rel = np.linalg.norm(a - b) / np.linalg.norm(a - u0)
    assert rel <= 1e-3, rel
    assert rel > 1e-8, rel          # the two schemes are distinct: K = 20 bursts are not K = 1
