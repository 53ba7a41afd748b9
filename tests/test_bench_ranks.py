"""bench.py on the CPU.  Multi-rank path: two gloo ranks agree on the slowest
rank's time, and every rank runs its own seeded replica of the benchmark
workload (same shape, distinct source amplitudes, rank 0 equal to the one-GPU
workload).  Reference arm: the oracle's line carries the contract's keys and
only rank 0 prints it."""
import hashlib
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _summary(amp):
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    return amp.shape, hashlib.sha256(amp.tobytes()).hexdigest(), float(amp.min()), float(amp.max())


def _rank_main(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench.dist_env()
        ms = bench.max_over_ranks(times[rank], tdist, "cpu")
        amp = np.asarray(bench.replica_workload(got_rank, got_ws)["src_amp"], dtype=np.float64)
        tdist.barrier()
        # a digest, not the array: a pipe holds only a few tens of KB before a put blocks
        out.put((rank, got_ws, got_local, ms, _summary(amp)))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_run_distinct_replicas():
    ws = 2
    times = [3.25, 7.5]
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, times, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(out.get() for _ in range(ws))
    assert [r[0] for r in res] == [0, 1]
    for rank, got_ws, got_local, ms, _ in res:
        assert got_ws == ws and got_local == rank
        assert ms == max(times)
    import bench
    single = _summary(bench.replica_workload(0, 1)["src_amp"])
    s0, s1 = res[0][4], res[1][4]
    assert s0[0] == s1[0] == single[0]
    assert s0[1] == single[1]                 # rank 0 runs the one-GPU workload itself
    assert s1[1] != s0[1]                     # rank 1 its own amplitudes
    assert s1[2] >= 0.5 and s1[3] <= 1.5


def test_max_over_ranks_without_a_group_is_the_identity():
    import bench
    assert bench.max_over_ranks(4.5, None, "cpu") == 4.5


def test_replicas_are_deterministic_and_keep_the_workload_shape():
    import bench
    a = bench.replica_workload(3, 4)
    b = bench.replica_workload(3, 4)
    one = bench.replica_workload(0, 1)
    np.testing.assert_array_equal(np.asarray(a["src_amp"]), np.asarray(b["src_amp"]))
    for key in ("n_xi", "n_eta", "m_xi", "m_eta", "k_micro", "n_macro"):
        assert a[key] == one[key], key


def _bench(args, env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                         env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    return lines


def _digest(probs):
    h = hashlib.sha256()
    for p in probs:
        h.update(repr(sorted((k, v) for k, v in p.items() if k != "src_amp")).encode())
    return h.hexdigest()


def test_batch_replicas_keep_the_recipe_and_differ_by_rank():
    import bench
    from paper_2405_08764_gb300 import workloads as W
    one = bench.replica_batch(0, 1)
    assert len(one) == 4096
    assert _digest(one) == _digest(W.c4_batch(4096))          # the one-GPU workload itself
    assert _digest(bench.replica_batch(0, 2)) == _digest(one)   # rank 0 of a launch runs it too
    r1 = bench.replica_batch(1, 2)
    assert len(r1) == 4096 and _digest(r1) != _digest(one)
    assert _digest(bench.replica_batch(1, 2)) == _digest(r1)
    for p in r1:
        assert p["n_xi"] in (16, 32, 64, 128) and p["m_xi"] in (5, 7, 9, 11) and p["k_micro"] == 20


def test_batch_update_count_and_accuracy_sample():
    import bench
    from paper_2405_08764_gb300 import workloads as W
    probs = W.c4_batch(64)
    n = bench.batch_updates(probs, 3)
    assert n == 3 * sum(W.n_patch(p) * p["m_xi"] ** 2 * 20 for p in probs)
    sel = bench.accuracy_sample(probs)
    assert sel == sorted(set(sel)) and sel[-1] == len(probs) - 1
    assert {probs[k]["map"] for k in sel} == {"identity", "tanh", "polar"}
    assert {probs[k]["m_xi"] for k in sel} == {5, 7, 9, 11}
    assert bench.flop_per_update(True) == 25.0 and bench.flop_per_update(False) == 20.0


def test_reference_arm_prints_one_contract_line_on_rank_0_only():
    lines = _bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--instances", "6"],
                   {"OMP_NUM_THREADS": "2"})
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["unit"] == d["e2e"]["unit"] == d["cpu_baseline"]["unit"]
    assert "workload" in d["config"]
    assert "4096" in d["config"]["workload"]
    # other ranks of a torchrun launch exit without work
    assert _bench(["--impl", "reference", "--steps", "1", "--warmup", "3"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
    # the 65x65 problem's reference line
    c2 = _bench(["--impl", "reference", "--workload", "c2", "--steps", "1", "--warmup", "1"], {"OMP_NUM_THREADS": "2"})
    assert len(c2) == 1 and "65x65" in c2[0]["config"]["workload"] and c2[0]["value"] > 0
