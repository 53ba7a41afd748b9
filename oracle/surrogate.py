"""Plain FP64 CPU oracle of the learned surrogate for the restricted macro time
derivative F (the patch scheme's (U^1 - U^0)/tau, eq. (Time_Derivative)).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's
CPU leg; the product library never imports it.  The paper has no surrogate;
the readings below define one so that it can be checked:

* features (35 per patch):
  - 25 stencil features: the 5x5 macro stencil U(i+p, j+q), p, q in -2..2
    (xi wraps on periodic grids, otherwise clamps; eta clamps to the boundary
    rows), taken through the tensor product of the 1-D difference basis
    e0 = u0, e1 = (u1 - u-1)/2, e2 = u1 - 2u0 + u-1,
    e3 = (u2 - 2u1 + 2u-1 - u-2)/2, e4 = u2 - 4u1 + 6u0 - 4u-1 + u-2
    (an invertible map of the 25 values), feature 5*q_ord + p_ord.  With s the
    largest magnitude of the 24 non-constant terms, term k >= 1 becomes D_k/s
    and the constant term U00/(|U00| + s);
  - 4 metric terms at the patch centre, each over the macro explicit rate R
    and times the stencil feature of the derivative it multiplies:
    2 alpha/(dxi^2 R) x[2], 2 gamma/(deta^2 R) x[10], nu/(dxi R) x[1],
    omega/(deta R) x[5], with
    R = 2 alpha/dxi^2 + 2 gamma/deta^2 + |beta|/(dxi deta) + |nu|/dxi + |omega|/deta + |phi|
    (the operator of Section 2, eq. (Computational_Problem));
  - 6 coefficient samples: half the trace of the diffusion tensor at the patch
    centre, its relative change at the four edge midpoints (xi +- h_xi/2,
    eta +- h_eta/2; order E, W, N, S), and tau * R;
* target y = F / (R s); the network sees standardised features (x - mu)/sigma
  and predicts y / y_scale;
* residual check: F1 is the restricted change of a one-micro-step burst
  (same micro step) over that step; F-hat is accepted when
  |F-hat - F1| <= eps (|F1| + rho), rho the RMS of F1 over the instance's
  patches, eps = 1e-3; otherwise the patch takes the full K-step burst;
* network: 35 -> 256 -> 256 -> 256 -> 1, GELU in its tanh form
  g(x) = x/2 (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))) (Hendrycks & Gimpel,
  2016), inputs padded to 64 with zeros.  Flat parameter layout (FP32 on the
  device, FP64 here): W1[256][64], b1[256], W2[256][256], b2[256],
  W3[256][256], b3[256], w4[256], b4.  On the device each standardised
  input x enters the first BF16 product as two terms, hi = bf16(x) and
  lo = bf16(x - hi) (x in FP32), both multiplied by bf16(W1).

Parity: the MLP backward is pinned by central finite differences and the GELU
by its odd-part identity; the features by exact discrete derivatives of
polynomials and scale invariance; the check and the surrogate step by their
definitions on small cases (see tests/test_oracle_surrogate.py).
"""
from __future__ import annotations

import math

import numpy as np

from . import Oracle

N_IN = 35
N_PAD = 64
WIDTH = 256
SHAPES = [("W1", (WIDTH, N_PAD)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("w4", (WIDTH,)), ("b4", (1,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


# ---------------------------------------------------------------------------
# parameters

def unflatten(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAM,)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in), fan_in = 35 for layer 1),
    zero biases, zero padding columns."""
    rng = np.random.default_rng(seed)
    p = {}
    b = math.sqrt(6.0 / N_IN)
    W1 = np.zeros((WIDTH, N_PAD))
    W1[:, :N_IN] = rng.uniform(-b, b, (WIDTH, N_IN))
    p["W1"] = W1
    b = math.sqrt(6.0 / WIDTH)
    p["W2"] = rng.uniform(-b, b, (WIDTH, WIDTH))
    p["W3"] = rng.uniform(-b, b, (WIDTH, WIDTH))
    p["w4"] = rng.uniform(-math.sqrt(3.0 / WIDTH), math.sqrt(3.0 / WIDTH), WIDTH)
    for k in ("b1", "b2", "b3"):
        p[k] = np.zeros(WIDTH)
    p["b4"] = np.zeros(1)
    return flatten(p)


# ---------------------------------------------------------------------------
# GELU (tanh form) and the MLP

def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GELU_C * (x + GELU_A * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * x * x)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even) through FP32, as the
    device's __float2bfloat16_rn does after an FP32 value is formed."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    r = np.where(np.isfinite(f), r, u)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def split_input(X):
    """hi + lo with hi = bf16(x) and lo = bf16(x - hi), x taken in FP32."""
    x32 = np.asarray(X, dtype=np.float32).astype(np.float64)
    hi = bf16(x32)
    lo = bf16((x32 - hi).astype(np.float32))
    return hi, lo


def forward(theta, X, round_bf16: bool = False):
    """y = w4 . g(W3 g(W2 g(W1 x + b1) + b2) + b3) + b4 for every row of X
    (X: [n, 64] or [n, 35]).  With round_bf16 the inputs enter as hi + lo
    (split_input), and W1..W3, w4 and the first two hidden activations are
    rounded to BF16 where the device rounds them (the third activation stays
    FP32 on the device)."""
    p = unflatten(theta)
    X = np.asarray(X, dtype=np.float64)
    if X.shape[1] == N_IN:
        X = np.pad(X, ((0, 0), (0, N_PAD - N_IN)))
    r = bf16 if round_bf16 else (lambda a: a)
    if round_bf16:
        hi, lo = split_input(X)
        z1 = (hi @ r(p["W1"]).T + lo @ r(p["W1"]).T) + p["b1"]
    else:
        z1 = X @ p["W1"].T + p["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ r(p["W2"]).T + p["b2"]
    h2 = r(gelu(z2))
    z3 = h2 @ r(p["W3"]).T + p["b3"]
    h3 = gelu(z3)
    y = h3 @ r(p["w4"]) + p["b4"][0]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss(theta, X, t):
    """Mean squared error (1/n) sum (y - t)^2."""
    y, _ = forward(theta, X)
    return float(np.mean((y - t) ** 2))


def gradient(theta, X, t, round_bf16: bool = False):
    """Gradient of loss() with respect to the flat parameters, by the chain
    rule through the four layers.  With round_bf16 the forward pass rounds as
    in forward(), and the back-propagated dZ of each layer is rounded to BF16
    before it enters the weight and input gradients (the device stores dZ in
    BF16 as a tensor-core operand); the bias gradients then sum the rounded dZ,
    and the first layer's weight gradient takes the high input part only."""
    p = unflatten(theta)
    r = bf16 if round_bf16 else (lambda a: a)
    y, c = forward(theta, X, round_bf16)
    n = len(t)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n
    g = {}
    g["w4"] = c["h3"].T @ dy
    g["b4"] = np.array([dy.sum()])
    dz3 = r(np.outer(dy, r(p["w4"])) * gelu_grad(c["z3"]))
    g["W3"] = dz3.T @ c["h2"]
    g["b3"] = dz3.sum(0)
    dz2 = r((dz3 @ r(p["W3"])) * gelu_grad(c["z2"]))
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = r((dz2 @ r(p["W2"])) * gelu_grad(c["z1"]))
    g["W1"] = dz1.T @ r(c["X"])
    g["b1"] = dz1.sum(0)
    return flatten(g)


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) with bias correction; step counts
    from 1.  Returns the new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# features

def basis_1d(u):
    """Difference basis of five equally spaced values u[..., 0..4] (offsets -2..2)."""
    um2, um1, u0, u1, u2 = (u[..., k] for k in range(5))
    return np.stack([u0, 0.5 * (u1 - um1), u1 - 2.0 * u0 + um1,
                     0.5 * (u2 - 2.0 * u1 + 2.0 * um1 - um2),
                     u2 - 4.0 * u1 + 6.0 * u0 - 4.0 * um1 + um2], -1)


def _patch_nodes(o: Oracle, sel):
    I, J = o.patch_nodes()
    return (I, J) if sel is None else (I[sel], J[sel])


def stencils(o: Oracle, U, sel=None):
    """The 5x5 macro stencil of every patch (or of the patches sel):
    [n, 5 (q: eta), 5 (p: xi)]."""
    s = o.s
    Ug = np.asarray(U, dtype=np.float64).reshape(o.nyp, o.nxp)
    I, J = _patch_nodes(o, sel)
    st = np.empty((len(I), 5, 5))
    for q in range(-2, 3):
        rows = np.clip(J + q, 0, s.n_eta)
        for p in range(-2, 3):
            cols = (I + p) % o.nxp if s.periodic_xi else np.clip(I + p, 0, s.n_xi)
            st[:, q + 2, p + 2] = Ug[rows, cols]
    return st


def stencil_features(st):
    """25 normalised difference-basis features and the scale s of each stencil."""
    a = basis_1d(st)                                  # along xi: [n, q, p_ord]
    b = basis_1d(np.swapaxes(a, 1, 2))                # along eta: [n, p_ord, q_ord]
    D = np.swapaxes(b, 1, 2).reshape(len(st), 25)     # feature 5*q_ord + p_ord
    s = np.abs(D[:, 1:]).max(1)
    x = np.zeros_like(D)
    nz = s > 0
    x[nz, 1:] = D[nz, 1:] / s[nz, None]
    den = np.abs(D[:, 0]) + s
    x[:, 0] = np.where(den > 0, D[:, 0] / np.where(den > 0, den, 1.0), 0.0)
    return x, s


def static_features(o: Oracle, sel=None):
    """Per-patch features that do not change with U: 4 metric terms, 6
    coefficient samples, and the rate R, of every patch or of the patches
    sel.  Returns (feat [n, 10], R [n])."""
    s = o.s
    dxi = (s.xi1 - s.xi0) / s.n_xi
    deta = (s.eta1 - s.eta0) / s.n_eta
    hx, hy = s.h_ratio_xi * dxi, s.h_ratio_eta * deta
    I, J = _patch_nodes(o, sel)
    xi = s.xi0 + I * dxi
    eta = s.eta0 + J * deta
    n = len(I)
    out = np.zeros((n, 10))
    R = np.zeros(n)
    tau = o.tau()

    def dhalf(a, b):
        m = o.map(a, b)
        ph = o.physical(m[0], m[1])
        return 0.5 * (ph[0] + ph[2])

    for k in range(n):
        al, be, ga, nu, om, ph = o.coeffs(xi[k], eta[k])[:6]
        r = 2 * al / dxi ** 2 + 2 * ga / deta ** 2 + abs(be) / (dxi * deta) + abs(nu) / dxi + abs(om) / deta + abs(ph)
        R[k] = r
        dc = dhalf(xi[k], eta[k])
        de = [dhalf(xi[k] + hx / 2, eta[k]), dhalf(xi[k] - hx / 2, eta[k]),
              dhalf(xi[k], eta[k] + hy / 2), dhalf(xi[k], eta[k] - hy / 2)]
        out[k] = [2 * al / (dxi ** 2 * r), 2 * ga / (deta ** 2 * r), nu / (dxi * r), om / (deta * r),
                  dc] + [(d - dc) / dc for d in de] + [tau * r]
    return out, R


def features(o: Oracle, U, static=None, sel=None):
    """Raw (unstandardised) features [n_patch, 35], the scale s and the rate R:
    the stencil features, the metric terms times the stencil feature of the
    derivative each multiplies (x[2] = xi-second, x[10] = eta-second,
    x[1] = xi-first, x[5] = eta-first difference), the coefficient samples."""
    fs, R = static_features(o, sel) if static is None else static
    x, s = stencil_features(stencils(o, U, sel))
    fs = fs.copy()
    fs[:, 0] *= x[:, 2]
    fs[:, 1] *= x[:, 10]
    fs[:, 2] *= x[:, 1]
    fs[:, 3] *= x[:, 5]
    return np.concatenate([x, fs], 1), s, R


def standardise(X, mu, sigma):
    return (X - mu) / sigma


# ---------------------------------------------------------------------------
# patch-solver targets, the residual check and the surrogate macro step

def patch_F(o: Oracle, U, t, k_micro=None):
    """F = restricted change / (k * dt) of every patch, from the plain FP64
    patch solver with k micro steps of the instance's micro step dt."""
    sel = np.arange(o.n_patch, dtype=np.int32)
    dt = o.dt_micro()
    if k_micro is None or k_micro == o.s.k_micro:
        return o.patch_dU(U, t, sel) / (o.s.k_micro * dt)
    o1 = Oracle(dict(o.prob, k_micro=int(k_micro)))
    return o1.patch_dU(U, t, sel, dt_micro=dt) / (k_micro * dt)


def check(F_hat, F1, eps=1e-3):
    """Accept mask of the residual check: |F_hat - F1| <= eps (|F1| + rms(F1)).
    A negative eps accepts nothing (every patch takes the burst), also where
    F_hat = F1 = 0 would meet the bound with equality."""
    if eps < 0:
        return np.zeros(len(F1), dtype=bool)
    rho = math.sqrt(float(np.mean(np.asarray(F1) ** 2))) if len(F1) else 0.0
    return np.abs(F_hat - F1) <= eps * (np.abs(F1) + rho)


def surrogate_F(o: Oracle, U, t, theta, mu, sigma, y_scale, static=None, round_bf16=False, eps=1e-3):
    """The surrogate's macro time derivative with the check and fallback.
    Returns (F, accepted mask, F_hat, F1)."""
    X, s, R = features(o, U, static)
    y, _ = forward(theta, standardise(X, mu, sigma), round_bf16)
    F_hat = y * y_scale * R * s
    F1 = patch_F(o, U, t, 1)
    ok = check(F_hat, F1, eps)
    F = F_hat.copy()
    if not ok.all():
        F[~ok] = patch_F(o, U, t)[~ok]
    return F, ok, F_hat, F1


def surrogate_step(o: Oracle, U, t0, dt_macro, n_steps, theta, mu, sigma, y_scale, round_bf16=False, eps=1e-3):
    """n macro steps of eq. (Extrapolation) with the surrogate's F; returns
    (U, number of fallback patches)."""
    static = static_features(o)
    U = np.array(U, dtype=np.float64)
    tau = o.tau()
    n_fb = 0
    for k in range(n_steps):
        t = t0 + k * dt_macro
        F, ok, _, _ = surrogate_F(o, U, t, theta, mu, sigma, y_scale, static, round_bf16, eps)
        n_fb += int((~ok).sum())
        U = o.project(U, F * tau, t, dt_macro, tau)
    return U, n_fb
