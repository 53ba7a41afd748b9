"""Planted mistakes in scratch copies of the oracle's Python modules (the
surrogate and the second-order integrators; CPU only): each must make at least
one of that module's pins fail.  The mutated module replaces the original in
a child interpreter that then runs the pins."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = {
    "surrogate": ["tests/test_oracle_surrogate.py"],
    "integrators": ["tests/test_oracle_integrators.py"],
}

MUTATIONS = {
    "gelu_cubic_dropped": ("surrogate", "return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))",
                           "return 0.5 * x * (1.0 + np.tanh(GELU_C * x))"),
    "basis_first_difference_sign": ("surrogate", "0.5 * (u1 - um1)", "0.5 * (um1 - u1)"),
    "stencil_transposed": ("surrogate", "st[:, q + 2, p + 2] = Ug[rows, cols]", "st[:, p + 2, q + 2] = Ug[rows, cols]"),
    "stencil_eta_wrapped": ("surrogate", "rows = np.clip(J + q, 0, s.n_eta)", "rows = (J + q) % (s.n_eta + 1)"),
    "metric_feature_index": ("surrogate", "fs[:, 0] *= x[:, 2]", "fs[:, 0] *= x[:, 10]"),
    "rate_cross_term_dropped": ("surrogate", "+ abs(be) / (dxi * deta) ", ""),
    "edge_samples_swapped": ("surrogate", "de = [dhalf(xi[k] + hx / 2, eta[k]), dhalf(xi[k] - hx / 2, eta[k]),",
                             "de = [dhalf(xi[k] - hx / 2, eta[k]), dhalf(xi[k] + hx / 2, eta[k]),"),
    "check_rho_dropped": ("surrogate", "return np.abs(F_hat - F1) <= eps * (np.abs(F1) + rho)",
                          "return np.abs(F_hat - F1) <= eps * np.abs(F1)"),
    "adam_bias_correction_dropped": ("surrogate", "mh = m / (1.0 - b1 ** step)", "mh = m"),
    "backward_transposed_weight": ("surrogate", 'g["W2"] = dz2.T @ c["h1"]', 'g["W2"] = c["h1"].T @ dz2'),
    "forward_bias_dropped": ("surrogate", 'z2 = h1 @ r(p["W2"]).T + p["b2"]', 'z2 = h1 @ r(p["W2"]).T'),
    "input_not_standardised": ("surrogate", "y, _ = forward(theta, standardise(X, mu, sigma), round_bf16)",
                               "y, _ = forward(theta, X, round_bf16)"),
    "fallback_takes_F1": ("surrogate", "F[~ok] = patch_F(o, U, t)[~ok]", "F[~ok] = F1[~ok]"),
    "surrogate_step_time_frozen": ("surrogate", "        t = t0 + k * dt_macro\n        F, ok, _, _ = surrogate_F(",
                                   "        t = t0\n        F, ok, _, _ = surrogate_F("),
    "negative_eps_accepts_zeros": ("surrogate", "    if eps < 0:\n        return np.zeros(len(F1), dtype=bool)\n", ""),
    "heun_stage_time": ("integrators", "F2 = patch_F(o, Us, t + dt)", "F2 = patch_F(o, Us, t)"),
    "ab2_history_sign": ("integrators", "(1.5 * F - 0.5 * F_prev)", "(1.5 * F + 0.5 * F_prev)"),
}

RUNNER = r'''
import importlib.util, sys
root, name, path = sys.argv[1], sys.argv[2], sys.argv[3]
sys.path.insert(0, root)
import oracle
spec = importlib.util.spec_from_file_location("oracle." + name, path)
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle." + name] = mod
spec.loader.exec_module(mod)
setattr(oracle, name, mod)
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider"] + sys.argv[4:]))
'''


def test_every_anchor_is_present_once():
    for name, (module, old, _) in MUTATIONS.items():
        src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
        assert src.count(old) == 1, name


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    module, old, new = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
    assert old in src, "mutation anchor missing: " + name
    path = tmp_path / (module + ".py")
    path.write_text(src.replace(old, new, 1))
    runner = tmp_path / "run_pins.py"
    runner.write_text(RUNNER)
    r = subprocess.run([sys.executable, str(runner), ROOT, module, str(path)] + PINS[module],
                       cwd=ROOT, capture_output=True, text=True)
    assert r.returncode not in (0, 4, 5), r.stdout[-2000:] + r.stderr[-2000:]
    assert r.returncode != 0, "planted mistake %s passed every pin:\n%s" % (name, r.stdout[-2000:])
