"""The seeded input generators (CPU): the five workloads have the stated
shapes and value ranges, and every draw is reproducible from its seed."""
import math

import numpy as np

from paper_2405_08764_gb300 import workloads as W


def test_configured_shapes():
    c1 = W.c1_manufactured()
    assert (c1["n_xi"], c1["m_xi"], c1["k_micro"], c1["n_macro"], c1["dt_macro"]) == (8, 7, 20, 50, 0.01)
    c2 = W.c2_heterogeneous()
    assert (c2["n_xi"], c2["n_eta"], c2["m_xi"], c2["k_micro"], c2["n_macro"], c2["map"]) == (64, 64, 11, 20, 200, "tanh")
    c3 = W.c3_annulus()
    assert (c3["n_eta"] + 1, c3["n_xi"], c3["m_xi"], c3["periodic_xi"], c3["map"]) == (128, 512, 9, 1, "polar")
    c5 = W.c5_surrogate_field()
    assert (c5["n_eta"] + 1, c5["n_xi"], c5["m_xi"], c5["periodic_xi"]) == (512, 2048, 9, 1)
    assert W.n_patch(c5) == 1044480
    b = W.bench_workload()
    np.testing.assert_array_equal(b.pop("src_amp"), c2.pop("src_amp"))
    assert b == c2


def test_batch_instances_are_reproducible_and_independent_of_the_batch_size():
    a, b = W.c4_batch(24), W.c4_batch(48)
    assert a == b[:24] == W.c4_batch(24)
    assert a[5] == W.c4_instance(5)
    assert a[5] != W.c4_instance(5, seed0=5)


def test_batch_instance_ranges():
    probs = W.c4_batch(256)
    assert {p["n_xi"] for p in probs} == {16, 32, 64, 128}
    assert {p["m_xi"] for p in probs} == {5, 7, 9, 11}
    assert {p["map"] for p in probs} == {"identity", "tanh", "polar"}
    for p in probs:
        m11, m12, m22 = p["M"]
        lam = np.linalg.eigvalsh(np.array([[m11, m12], [m12, m22]]))
        assert 1e-4 * (1 - 1e-12) <= lam[0] <= lam[1] <= 1e-1 * (1 + 1e-12)
        assert -2.0 <= p["va"][0] <= 2.0 and -2.0 <= p["vb"][0] <= 2.0 and 0.0 <= p["f0"] <= 1.0
        if p["map"] == "tanh":
            assert 1.0 <= p["map_p"][0] <= 4.0
        if p["map"] == "polar":
            assert 0.5 <= p["map_p"][0] <= 1.0 and 1.5 <= p["map_p"][1] <= 3.0 and p["periodic_xi"] == 1


def test_source_amplitudes_per_patch():
    p, q = W.c2_heterogeneous(), W.c2_heterogeneous(seed=3)
    amp = np.asarray(p["src_amp"])
    assert amp.shape == (W.n_patch(p),)
    assert amp.min() >= 0.5 and amp.max() <= 1.5
    np.testing.assert_array_equal(amp, W.c2_heterogeneous()["src_amp"])
    assert not np.array_equal(amp, q["src_amp"])


def test_annulus_fields_stay_positive_and_seeded():
    for seed in (5, 1000, 1007):
        p = W.c5_surrogate_field(n_r=7, n_theta=16, seed=seed)
        c = np.asarray(p["four"]["c"])
        assert len(c) == 3 and np.abs(c).max() <= 0.1        # D = 1 + sum c_k ... >= 0.7
        amps = np.asarray(p["init_p"][3:])
        assert len(amps) == 4 and amps.min() >= 0.5 and amps.max() <= 1.5
    a3 = np.asarray(W.c3_annulus()["init_p"][3:])
    assert a3.min() >= 0.5 and a3.max() <= 1.5 and math.isclose(W.c3_annulus()["map_p"][2], 1.5)
