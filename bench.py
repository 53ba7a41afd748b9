"""Benchmark of the patch-dynamics hot path on GB300.

Default workload (the largest single-GPU configuration): 4096 independent,
uneven constant-coefficient CDR instances (macro grids of 17..129 nodes per
side, identity / tanh-stretched / annular maps, 5x5..11x11 micro points per
patch, tensor diffusion with a cross term, K = 20 forward-Euler micro steps
per burst), all stepped together by the batched work-queue kernels, FP32
bursts with FP64 restriction and projection.  One bench step = one pd_step
call of 10 macro steps over every instance (lift -> burst -> restrict ->
project per macro step, captured in a CUDA graph) with the macro fields
already resident in HBM (182 MB of FP64 fields, larger than the L2, which is
also flushed between timed steps).  The same line carries the end-to-end
figure (host fields copied in and out every step), the error against the FP64
CPU oracle on sampled instances, the FP64 batch, and the 65x65 heterogeneous
problem on the persistent dataflow kernel.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload c4|c2|c5|passes|adi|refresh]
For N > 1 launch with torch.distributed.run: every rank runs an independent
replica of the workload on its own GPU (no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "patch point-updates/s (roofline frac), macro steps/s at fixed L2 err vs FP64"
UNIT = "point-updates/s"
N_INST = 4096
C4_MACRO = 10                 # macro steps per bench step of the batch workload
C4_WORKLOAD = ("4096 uneven constant-coefficient CDR instances (N in {16,32,64,128}, m in {5,7,9,11}, "
               "identity/tanh/annulus maps, rotated tensor D, K=20), 10 macro steps per step")
C2_WORKLOAD = "tanh-stretched heterogeneous CDR, 65x65 macro grid, 11x11 micro, K=20, 200 macro steps"


def flop_per_update(has_cross: bool) -> float:
    """Algorithmic FP32 flops of one point-update of the 9-point micro stencil:
    25 with the mixed-derivative (cross) term, 20 without it."""
    return 25.0 if has_cross else 20.0


# DRAM traffic of the dominant kernel from an ncu capture of this kernel
# source (sha256 of the sources); null once the kernel changes.
# For the batch: the eight launches of one macro step of the 4096-instance batch
# (four micro sizes, separable-map and other patch groups; profiles/batch_kernel_c4.md).
NCU_TRAFFIC = {"sources_sha256": "af0c707261038e2a9fdda8058bb1cd9f47c61603f1698010f72fa4d7625fe8a8",
               "bytes_per_launch": 455.7e6}


def kernel_sources_sha(files=("pd_batch.cu", "pd_device.cuh", "pd_internal.h")) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2405_08764_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peaks(device=None) -> dict:
    """Measured HBM and BF16 peaks (MEASURED_PEAKS.json, else the fallback
    figures) and the FP32 FMA peak from the device's SM count and the maximum
    SM clock."""
    p = {"hbm_gbs": None, "sm_max_mhz": 2070.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        p.update(hbm_gbs=d.get("hbm_gbs"), sm_max_mhz=d.get("sm_max_mhz", 2070.0), source="measured",
                 bf16_tflops=d.get("bf16_tflops", 1900.0))
    else:
        p["hbm_gbs"] = 6800.0
        p["bf16_tflops"] = 1900.0
    n_sm, sm_src = 152, "GB300 SM count"
    try:
        import torch
        if torch.cuda.is_available():
            dev = torch.cuda.current_device() if device is None else device
            n_sm, sm_src = torch.cuda.get_device_properties(dev).multi_processor_count, "device attribute"
    except Exception:
        pass
    p["n_sm"] = n_sm
    # FP32 FMA pipe: SMs x 128 lanes x 2 flop per clock at the maximum SM clock
    p["fp32_tflops"] = n_sm * 128 * 2 * p["sm_max_mhz"] * 1e6 / 1e12
    p["fp32_source"] = "%d SMs (%s) x 128 FP32 lanes x 2 flop x %.0f MHz (%s sm_max_mhz)" % (
        n_sm, sm_src, p["sm_max_mhz"], p["source"])
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# workloads of the ranks


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_batch(rank: int, ws: int, n_inst: int = N_INST) -> list:
    """The batch of one rank: the 4096-instance workload itself on rank 0 (and
    on one GPU); every other rank an independent batch of the same recipe
    drawn from its own seeds (weak scaling, no data-path collective)."""
    from paper_2405_08764_gb300 import workloads as W
    seed0 = 4 if rank == 0 else 4 + n_inst * rank
    return W.c4_batch(n_inst, seed0=seed0)


def replica_workload(rank: int, ws: int) -> dict:
    """The 65x65 heterogeneous problem of one rank: the problem itself on rank
    0; other ranks the same problem with their own seeded per-patch source
    amplitudes."""
    from paper_2405_08764_gb300 import workloads as W
    return W.bench_workload() if rank == 0 else W.c2_heterogeneous(seed=2 + rank)


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); ms unchanged without a group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def batch_updates(probs: list, n_macro: int) -> int:
    """Point-updates of n_macro macro steps over every instance, from the
    workload parameters: patches x micro points x K."""
    from paper_2405_08764_gb300 import workloads as W
    return sum(W.n_patch(p) * p["m_xi"] * p["m_eta"] * p["k_micro"] for p in probs) * n_macro


def accuracy_sample(probs: list) -> list:
    """Instances checked against the oracle: the first of every (map, micro
    size) pair, the first of the largest (N = 128, m = 11), the last one."""
    sel = []
    for mp in ("identity", "tanh", "polar"):
        for m in (5, 7, 9, 11):
            k = next((k for k, p in enumerate(probs) if p["map"] == mp and p["m_xi"] == m), None)
            if k is not None:
                sel.append(k)
    k = next((k for k, p in enumerate(probs) if p["n_xi"] == 128 and p["m_xi"] == 11), None)
    if k is not None:
        sel.append(k)
    sel.append(len(probs) - 1)
    return sorted(set(sel))


# --------------------------------------------------------------------------
# CPU baselines (the oracle as it stands, on the host cores)


def cpu_baseline(prob: dict, target_s: float = 12.0) -> dict:
    """The CPU oracle on a bounded sample of the 65x65 problem: macro steps from
    the initial field in chunks of 20 until about target_s seconds of CPU work
    (one untimed chunk first)."""
    import oracle
    o = oracle.Oracle(prob)
    U0 = o.init_field()
    dtm = 0.5 * o.dt_macro()
    dt = o.dt_micro()
    per_step = o.n_patch * o.mx * o.my * o.s.k_micro
    chunk = 20
    o.step(U0, 0.0, dtm, chunk, dt)
    total = 0
    t = time.perf_counter()
    while time.perf_counter() - t < target_s:
        o.step(U0, 0.0, dtm, chunk, dt)
        total += chunk
    el = time.perf_counter() - t
    return {"value": total * per_step / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d macro steps of the 65x65 problem in chunks of %d from the initial field (%.1f s)"
                      % (total, chunk, el)}


class OracleBatch:
    """The oracle over a fixed subset of the batch: each call advances every
    instance of the subset by one macro step (at its own suggested step)."""

    def __init__(self, probs: list):
        import oracle
        self.state = []
        for p in probs:
            o = oracle.Oracle(p)
            self.state.append([o, o.init_field(), o.dt_macro(), o.dt_micro(), 0.0])
        self.updates_per_round = sum(s[0].n_patch * s[0].mx * s[0].my * s[0].s.k_micro for s in self.state)

    def round(self):
        for s in self.state:
            o, U, dtm, dt, t = s
            s[1] = o.step(U, t, dtm, 1, dt)
            s[4] = t + dtm


def cpu_baseline_batch(probs: list, target_s: float = 12.0) -> dict:
    """The CPU oracle on the first 64 instances of the batch: rounds of one
    macro step of each instance until about target_s seconds of CPU work (one
    untimed round first), reported per point-update."""
    import oracle
    ob = OracleBatch(probs)
    ob.round()
    n = 0
    t = time.perf_counter()
    while time.perf_counter() - t < target_s or n == 0:
        ob.round()
        n += 1
    el = time.perf_counter() - t
    return {"value": n * ob.updates_per_round / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d rounds of one macro step of each of the first %d instances of the batch (%.1f s)"
                      % (n, len(probs), el)}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the paper publishes no code),
    timed as it stands on the host cores on a bounded sample of the same
    workload; rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    if args.workload == "c2":
        from paper_2405_08764_gb300 import workloads as W
        prob = W.bench_workload()
        o = oracle.Oracle(prob)
        U = o.init_field()
        dtm, dt = 0.5 * o.dt_macro(), o.dt_micro()
        per_round = o.n_patch * o.mx * o.my * o.s.k_micro * 20

        def one(s):
            nonlocal U
            U = o.step(U, s * 20 * dtm, dtm, 20, dt)
        sample = "20 of the 200 macro steps of the 65x65 problem per step"
        workload = C2_WORKLOAD
    else:
        ob = OracleBatch(replica_batch(0, 1)[:min(64, args.instances)])
        per_round = ob.updates_per_round

        def one(s):
            ob.round()
        sample = "one macro step of each of the first %d instances of the batch per step" % len(ob.state)
        workload = C4_WORKLOAD
    for s in range(args.warmup):
        one(s)
    el = 0.0
    for s in range(args.steps):
        t = time.perf_counter()
        one(args.warmup + s)
        el += time.perf_counter() - t
    value = args.steps * per_round / el
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload, "sample": sample, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%s, %d steps" % (sample, args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# the batch workload (default line)


def _rel_l2(a, b) -> float:
    import numpy as np
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def batch_oracle_error(g, probs, U0h, Uh, n_macro, sel) -> dict:
    """Relative L2 distance of the GPU fields from the FP64 oracle after
    n_macro macro steps (each instance at its suggested step) on the sampled
    instances."""
    import oracle
    errs = {}
    for k in sel:
        i = g.info(k)
        a, n = i["u_offset"], i["n_macro"]
        o = oracle.Oracle(probs[k])
        want = o.step(U0h[a:a + n], 0.0, o.dt_macro(), n_macro)
        errs[k] = _rel_l2(Uh[a:a + n], want)
    return {"max": max(errs.values()), "instances": len(errs),
            "per_instance": {str(k): v for k, v in errs.items()}}


def time_steps(g, U, U0, n_macro, steps, flush, stream):
    """K bench steps of n_macro macro steps, CUDA events on the launching
    stream around each, the field reset and the L2 flushed outside them."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s in range(steps):
        U.copy_(U0)
        flush.fill_(float(s))
        ev[s][0].record(stream)
        g.step(U, 0.0, 0.0, n_macro)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def time_e2e(g, U0, n_macro, steps, stream):
    """End to end through the public API: every step copies the host fields
    (pinned) to the device, runs pd_step and copies the result back; one
    untimed step first (graph capture for the new field pointer)."""
    import torch
    Uh = U0.cpu().pin_memory()
    Uout = torch.empty_like(Uh).pin_memory()
    Ud = torch.empty_like(U0)
    Ud.copy_(Uh, non_blocking=True)
    g.step(Ud, 0.0, 0.0, n_macro)
    Uout.copy_(Ud, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        Ud.copy_(Uh, non_blocking=True)
        g.step(Ud, 0.0, 0.0, n_macro)
        Uout.copy_(Ud, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), U0.numel() * 8


def batch_fp64(probs, n_macro, steps, sel, U0h) -> dict:
    """The same batch with FP64 bursts (the parity precision): time per bench
    step and error against the oracle."""
    import torch
    from paper_2405_08764_gb300.api import Grid
    g = Grid(probs, prec="fp64")
    U0 = g.init_field()
    U = U0.clone()
    g.step(U, 0.0, 0.0, n_macro)         # autotune + capture
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ms = time_steps(g, U, U0, n_macro, steps, flush, stream)
    g.sync()
    upd = batch_updates(probs, n_macro)
    U.copy_(U0)
    g.step(U, 0.0, 0.0, n_macro)
    g.sync()
    err = batch_oracle_error(g, probs, U0h, U.cpu().numpy(), n_macro, sel)
    return {"value": upd * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "dtype": "f64", "l2_rel_err_vs_oracle": err["max"]}


def run_batch(args):
    import numpy as np
    import torch

    from paper_2405_08764_gb300.api import Grid

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    probs = replica_batch(rank, ws, args.instances)
    n_macro = args.macro
    t = time.perf_counter()
    g = Grid(probs, prec=args.prec)
    setup_s = time.perf_counter() - t
    updates = batch_updates(probs, n_macro)
    n_cross = sum(1 for k in range(len(probs)) if g.info(k)["has_cross"])
    flop_step = sum(flop_per_update(g.info(k)["has_cross"]) * g.info(k)["n_patch"] * g.info(k)["m_xi"]
                    * g.info(k)["m_eta"] * g.info(k)["k_micro"] for k in range(len(probs)))
    U0 = g.init_field()
    U = U0.clone()
    field_bytes = U0.numel() * 8
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    t = time.perf_counter()
    U.copy_(U0)
    g.step(U, 0.0, 0.0, n_macro)      # autotune + capture + one run
    g.sync()
    first_s = time.perf_counter() - t
    for _ in range(max(0, args.warmup - 1)):
        U.copy_(U0)
        g.step(U, 0.0, 0.0, n_macro)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    g.set_timing(True)
    l0 = g.launches()
    torch.cuda.nvtx.range_push("timed")          # profilers can restrict a capture to this range
    ms = time_steps(g, U, U0, n_macro, args.steps, flush, stream)
    torch.cuda.nvtx.range_pop()
    launches = g.launches() - l0
    kern_ms, kern_n = g.timing()
    g.set_timing(False)
    clocks = sampler.stop()
    g.sync()
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    total_updates = sum_over_ranks(float(updates), dist, "cuda")
    value = total_updates * args.steps / (ms / 1e3)
    e2e_ms, nbytes = time_e2e(g, U0, n_macro, args.steps, stream)
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    e2e = total_updates * args.steps / (e2e_ms / 1e3)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    pk = peaks(local)
    # the dominant kernels: the batched macro-step kernels of one macro step
    # (per micro size, run concurrently); event time of the captured graph
    # launches divided by their macro steps
    per_macro_s = kern_ms / kern_n / 1e3 if kern_n else ms / 1e3 / (args.steps * n_macro)
    achieved = flop_step / per_macro_s / 1e12
    sha = kernel_sources_sha()
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["sources_sha256"] == sha else None
    U.copy_(U0)
    g.step(U, 0.0, 0.0, n_macro)
    g.sync()
    U0h, Uh = U0.cpu().numpy(), U.cpu().numpy()
    sel = accuracy_sample(probs)
    err32 = batch_oracle_error(g, probs, U0h, Uh, n_macro, sel)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": C4_WORKLOAD if len(probs) == N_INST else
                   C4_WORKLOAD.replace("4096", str(len(probs))),
                   "instances": len(probs), "macro_steps_per_step": n_macro,
                   "point_updates_per_step": updates, "instances_with_cross_term": n_cross,
                   "field_bytes": field_bytes, "setup_s": setup_s, "first_step_s": first_s,
                   "l2": "inputs larger than L2 (182 MB of fields) and L2 flushed between timed steps (512 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "macro_steps_per_s": n_macro * args.steps / (ms / 1e3),
        "l2_rel_err_vs_oracle": err32["max"],
        "accuracy": {"vs": "FP64 CPU oracle, %d macro steps from the initial fields" % n_macro,
                     "sampled_instances": err32["instances"], "max_rel_l2": err32["max"]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / pk["fp32_tflops"], "traffic": traffic,
                     "traffic_note": ("dram read + write of the four per-size launches of one macro step "
                                      "(the unit of achieved), one ncu capture of this kernel source on the "
                                      "4096-instance batch" if traffic is not None else
                                      "no DRAM capture of the current kernel source; the batch is ALU-bound "
                                      "(per macro step it reads and writes the FP64 fields, 2 x %.0f MB, and "
                                      "the 1-D metric tables)" % (field_bytes / 1e6)),
                     "kernel": "batch_kernel (work queue per micro size, one launch per micro size and macro step)",
                     "flop_per_macro_step": flop_step,
                     "flop_per_point_update": "25 with a cross term, 20 without (%d of %d instances have one)"
                                              % (n_cross, len(probs)),
                     "kernel_ms_per_macro_step": 1e3 * per_macro_s,
                     "peak_source": pk["fp32_source"]},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if ws == 1 and not args.no_extras:
        del g, U, U0, flush
        torch.cuda.empty_cache()
        line["fp64_batch"] = batch_fp64(probs, n_macro, max(1, min(2, args.steps)), sel, U0h)
        torch.cuda.empty_cache()
        line["c2"] = run_c2(args, extra=True)
    if ws == 1 and not args.no_cpu_baseline:      # the host baseline is a one-GPU figure
        line["cpu_baseline"] = cpu_baseline_batch(probs[:64])
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# the 65x65 heterogeneous problem (persistent dataflow kernel)


def run_c2(args, extra: bool = False):
    """The 65x65 tanh-stretched heterogeneous tensor-diffusion problem, 11x11
    micro points, 200 macro steps per bench step on the persistent dataflow
    kernel.  extra=True returns a summary dict for the batch line instead of
    printing a line of its own."""
    import numpy as np
    import torch

    from paper_2405_08764_gb300.api import Grid

    ws, rank, local = dist_env()
    if extra:
        ws, rank = 1, 0
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prob = replica_workload(rank, ws)
    g = Grid(prob, prec="fp32")
    info = g.info()
    n_macro = prob["n_macro"]
    dtm = info["dt_macro_suggested"]
    fpu = flop_per_update(info["has_cross"])
    updates = info["n_patch"] * info["m_xi"] * info["m_eta"] * info["k_micro"] * n_macro
    U0 = g.init_field()
    U = U0.clone()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    steps = args.steps
    for _ in range(args.warmup):
        U.copy_(U0)
        g.step(U, 0.0, dtm, n_macro)
    g.sync()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if not extra:
        sampler.start()
        time.sleep(0.3)
    g.set_timing(True)
    l0 = g.launches()
    for s in range(steps):
        U.copy_(U0)
        flush.fill_(float(s))
        ev[s][0].record(stream)
        g.step(U, 0.0, dtm, n_macro)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    launches = g.launches() - l0
    kern_ms, kern_n = g.timing()
    g.set_timing(False)
    clocks = sampler.stop() if not extra else None
    g.sync()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, "cuda")
    if dist:
        dist.barrier()
    value = ws * updates * steps / (ms / 1e3)

    Uh = U0.cpu().pin_memory()
    Uout = torch.empty_like(Uh).pin_memory()
    Ud = torch.empty_like(U0)
    Ud.copy_(Uh, non_blocking=True)
    g.step(Ud, 0.0, dtm, n_macro)        # graph capture for the new field pointer
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        Ud.copy_(Uh, non_blocking=True)
        g.step(Ud, 0.0, dtm, n_macro)
        Uout.copy_(Ud, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    e2e = ws * updates * steps / (e2e_ms / 1e3)
    nbytes = U0.numel() * 8

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # accuracy: FP32 and FP64 GPU results against the FP64 CPU oracle
    import oracle
    o = oracle.Oracle(prob)
    want = o.step(U0.cpu().numpy(), 0.0, dtm, n_macro)
    U.copy_(U0)
    g.step(U, 0.0, dtm, n_macro)
    g.sync()
    g64 = Grid(prob, prec="fp64")
    V = g64.init_field()
    g64.step(V, 0.0, dtm, n_macro)
    g64.sync()
    err = {"fp32": _rel_l2(U.cpu().numpy(), want), "fp64": _rel_l2(V.cpu().numpy(), want)}

    pk = peaks(local)
    per_launch_updates = updates / n_macro
    achieved = (fpu * per_launch_updates * kern_n / (kern_ms / 1e3)) / 1e12 if kern_ms > 0 else None
    sha = kernel_sources_sha(("pd_persist.cu", "pd_device.cuh", "pd_internal.h"))
    traffic = None
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
        "frac": (achieved / pk["fp32_tflops"]) if achieved else None, "traffic": traffic,
        "traffic_note": "no DRAM capture of this kernel: ncu fails the cooperative launch before it runs; a cold "
                        "launch reads the 30.7 MB of burst records once, later steps find them in L2",
        "kernel": ("patch_persist_kernel<11,cross,tsrc,float> (cooperative, %d macro steps per launch)"
                   % info["chunk_steps"] if info["exec_path"] == 2 else
                   "patch_warp_kernel<11,cross,tsrc,float,fused> (one macro step per launch)"),
        "flop_per_point_update": fpu,
        "kernel_ms_per_macro_step": kern_ms / kern_n if kern_n else None,
        "peak_source": pk["fp32_source"],
        "sources_sha256": sha[:16],
    }
    if extra:
        return {"workload": C2_WORKLOAD, "value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
                "macro_steps_per_s": n_macro * steps / (ms / 1e3), "l2_rel_err_vs_oracle": err,
                "roofline": roofline, "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                                              "d2h_bytes_per_step": nbytes}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C2_WORKLOAD, "macro_steps_per_step": n_macro, "n_patch": info["n_patch"],
                   "point_updates_per_step": updates, "dt_macro": dtm,
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "macro_steps_per_s": n_macro * steps / (ms / 1e3),
        "l2_rel_err_vs_oracle": err["fp32"],
        "l2_rel_err_vs_oracle_fp64_path": err["fp64"],
        "roofline": roofline,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(prob)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# other workloads


def run_surrogate(args):
    """Annulus 512 radial x 2048 angular nodes, 9x9 micro, seeded smooth D:
    the surrogate-accelerated scheme (network trained here on the GPU from
    patch-solver data of 8 other seeded fields, 2.1e6 samples) against the
    plain FP64 and FP32 schemes, 100 macro steps each, same grid and steps."""
    import numpy as np
    import torch

    from paper_2405_08764_gb300 import workloads as W
    from paper_2405_08764_gb300.api import MLP, Grid, Surrogate

    torch.cuda.set_device(0)
    n_macro = 100
    n_r, n_theta = (int(v) for v in args.c5_grid.split("x"))
    p = W.c5_surrogate_field(n_r=n_r, n_theta=n_theta)
    # training data from the patch solver: fields at step 0 and step 50, each also
    # with 4 grid-scale perturbations (relative size 1e-10..1e-5), every 40th patch
    t0 = time.perf_counter()
    net = MLP(4096)
    rng = np.random.default_rng(8)
    Xs, ys = [], []
    for sd in range(1000, 1008):
        q = W.c5_surrogate_field(n_r=n_r, n_theta=n_theta, seed=sd)
        g = Grid(q, prec="fp32")
        s = Surrogate(g, net)
        U = g.init_field()
        dtm = g.info()["dt_macro_suggested"]
        for k in range(2):
            for c in range(5):
                V = U if c == 0 else s.perturb(U, 10.0 ** rng.uniform(-10, -5), int(rng.integers(1 << 62)))
                f = s.features(V, standardised=False, raw=True)
                y = s.targets(V, k * 50 * dtm, f["Rs"])
                o = int(rng.integers(40))
                Xs.append(f["X_raw"][o::40].contiguous())
                ys.append(y[o::40].contiguous())
            g.step(U, k * 50 * dtm, dtm, 50)
        del s, g
    Xr, yr = torch.cat(Xs), torch.cat(ys)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    net.fit_norm(Xr, yr)
    X, tt = net.pack(Xr, yr)
    net.init(21)
    t0 = time.perf_counter()
    hist = net.train(X, tt, batch=args.batch, epochs=args.epochs, lr_max=2e-3, seed=2)
    net.sync()
    train_s = time.perf_counter() - t0
    n_train = int(X.shape[0])

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(torch.cuda.current_stream())
        fn()
        b.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    res = {}
    fields = {}
    # plain_k1: the plain scheme with bursts of one micro step (tau = dt_micro),
    # i.e. the residual check's own estimator F1 run as the scheme
    for name, prec, k in (("plain_fp64", "fp64", None), ("plain_fp32", "fp32", None),
                          ("plain_k1_fp32", "fp32", 1), ("plain_k1_fp64", "fp64", 1)):
        g = Grid(p if k is None else dict(p, k_micro=k), prec=prec)
        dtm = g.info()["dt_macro_suggested"]
        U = g.init_field()
        g.step(U.clone(), 0.0, dtm, 2)          # warm-up (graph capture for 2 steps)
        res[name] = timed(lambda: g.step(U, 0.0, dtm, n_macro))
        g.sync()
        fields[name] = U
    g = Grid(p, prec="fp32")
    s = Surrogate(g, net)
    dtm = g.info()["dt_macro_suggested"]
    W_ = g.init_field()
    s.step(W_, 0.0, dtm, 2)                      # warm-up
    U = g.init_field()
    # the method without the network: every patch takes the one-step estimate F1
    W1 = g.init_field()
    s.step_f1(W1.clone(), 0.0, dtm, 2)           # warm-up
    res["f1_only"] = timed(lambda: s.step_f1(W1, 0.0, dtm, n_macro))
    fields["f1_only"] = W1
    st0, fb0 = s.counts()
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.nvtx.range_push("surrogate_steps")
    res["surrogate"] = timed(lambda: s.step(U, 0.0, dtm, n_macro, eps=1e-3))
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    g.sync()
    st1, fb1 = s.counts()
    fields["surrogate"] = U
    # the network forward alone over every patch (the dominant kernel of the step)
    Xf = s.features(U)["X"]
    yf = net.forward(Xf)
    n_rows = int(Xf.shape[0])
    reps = 5
    t_fwd = timed(lambda: [net.forward(Xf, out=yf) for _ in range(reps)]) / reps
    flop_row = 2.0 * (35 * 256 + 256 * 256 + 256 * 256 + 256)     # algorithmic: 35-256-256-256-1
    achieved = flop_row * n_rows / t_fwd / 1e12
    pk = peaks()
    ref = fields["plain_fp64"]
    err = {k: (torch.linalg.norm(v - ref) / torch.linalg.norm(ref)).item() for k, v in fields.items() if k != "plain_fp64"}
    served = 1.0 - (fb1 - fb0) / max(1, st1 - st0)
    value = n_macro / res["surrogate"]
    line = {
        "metric": METRIC, "value": value, "unit": "macro steps/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * res["surrogate"] / n_macro, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
        "config": {"workload": "annulus %dx%d macro nodes, 9x9 micro, K=20, seeded smooth D, 100 macro steps; "
                               "surrogate 35-256-256-256-1 trained on %d patch-solver samples of 8 other fields"
                               % (n_r + 1, n_theta, n_train),
                   "training_data": "8 seeded fields x 2 times x (clean + 4 perturbed) x every 40th patch",
                   "train_epochs": args.epochs, "train_batch": args.batch, "train_s": train_s, "data_s": data_s,
                   "loss_first_last": [float(hist[0]), float(hist[-1])], "check_eps": 1e-3},
        "macro_steps_per_s": {k: n_macro / v for k, v in res.items()},
        "speedup_vs_plain_fp64": res["plain_fp64"] / res["surrogate"],
        "speedup_vs_plain_fp32": res["plain_fp32"] / res["surrogate"],
        "speedup_vs_plain_k1_fp32": res["plain_k1_fp32"] / res["surrogate"],
        "speedup_vs_f1_only": res["f1_only"] / res["surrogate"],
        "l2_rel_vs_plain_fp64": err,
        "served_by_network": served,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / pk["bf16_tflops"], "traffic": None,
                     "kernel": "mlp_fused_kernel (network forward over %d patches: three tcgen05 BF16 layers "
                               "per 128-row tile on chip, one persistent block per SM)" % n_rows,
                     "flop_per_row": flop_row, "ms": 1e3 * t_fwd,
                     "peak_source": "measured cuBLAS bf16 burst"},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_passes(args):
    """The separate C-ABI passes (pd_lift, pd_micro_burst, pd_restrict, pd_project)
    timed one by one on the 512x2048-node annulus (84.6 M micro points), L2
    flushed before every timed pass; HBM-bound passes against the measured
    copy bandwidth, the burst against the FP32 ALU peak."""
    import torch

    from paper_2405_08764_gb300 import workloads as W
    from paper_2405_08764_gb300.api import Grid

    torch.cuda.set_device(0)
    n_r, n_theta = (int(v) for v in args.c5_grid.split("x"))
    p = W.c5_surrogate_field(n_r=n_r, n_theta=n_theta)
    g = Grid(p, prec="fp32")
    info = g.info()
    P, m, K = info["n_patch"], info["m_xi"], info["k_micro"]
    pts = P * m * m
    es = 4                                   # FP32 grid
    U = g.init_field()
    dtm = info["dt_macro_suggested"]
    st = g.new_state()
    dU = torch.empty(P, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5):
        tot = 0.0
        for r in range(reps + 1):
            flush.fill_(float(r))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                tot += a.elapsed_time(b)
        return tot / reps / 1e3

    n_int = P                                # interior macro nodes = patches
    bytes_ = {
        # per micro point: the FP32 coefficient record (32 B) in, u0 (8 B) + r + w (2 x 4 B) out;
        # per patch: 9 stencil reads (cached), edge data 4 (m + 2) x 8 B and the bias out
        "lift": pts * (32 + 8 + 2 * es) + P * (4 * (m + 2) * 8 + 8),
        # per micro point: w and r in (K steps in registers), w out; burst record (64 B) in
        "burst": pts * (2 * es + es + 64),
        # per micro point w in; per patch bias in, dU out
        "restrict": pts * es + P * 16,
        # per interior node U and dU in, U out
        "project": n_int * 24,
    }
    calls = {
        "lift": lambda: g.lift(U, 0.0, st),
        "burst": lambda: g.micro_burst(st, 0.0, K),
        "restrict": lambda: g.restrict(st, dU),
        "project": lambda: g.project(U, dU, 0.0, 1e-12),
    }
    for fn in calls.values():
        fn()
    torch.cuda.synchronize()
    pk = peaks()
    sampler = ClockSampler(0)
    sampler.start()
    res = {}
    for name, fn in calls.items():
        s = timed(fn)
        gbs = bytes_[name] / s / 1e9
        res[name] = {"ms": 1e3 * s, "bytes": bytes_[name], "GB_per_s": gbs, "frac_hbm": gbs / pk["hbm_gbs"]}
    clocks = sampler.stop()
    upd = pts * K
    res["burst"]["point_updates_per_s"] = upd / (res["burst"]["ms"] / 1e3)
    res["burst"]["frac_fp32"] = flop_per_update(info["has_cross"]) * res["burst"]["point_updates_per_s"] / 1e12 / pk["fp32_tflops"]
    line = {
        "metric": "separate C-ABI passes: achieved HBM GB/s (lift, restrict, project), burst point-updates/s",
        "value": res["lift"]["GB_per_s"], "unit": "GB/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "annulus %dx%d macro nodes, %dx%d micro, K=%d: %d micro points" % (n_r + 1, n_theta, m, m, K, pts),
                   "l2": "flushed before every timed pass (512 MB write)", "reps": 5},
        "passes": res, "hbm_peak_gbs": pk["hbm_gbs"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_adi(args):
    """Section 4.1.1 at the paper's patch settings (h = 1e-3, n = 10 nano
    intervals, bursts of tau = 1e-6 made of n_t = 2 ADI steps, lambda = 0.1) on
    an N x N macro grid, FP32 bursts: one bench step = 20 macro steps through
    pd_step (one ADI kernel per macro step, graph-captured), L2 flushed between
    steps.  Beside it the same bursts made of forward-Euler steps (K = tau / dt
    at the explicit bound) on the same grid."""
    import numpy as np
    import torch

    from paper_2405_08764_gb300 import workloads as W
    from paper_2405_08764_gb300.api import Grid

    torch.cuda.set_device(0)
    n = args.adi_n
    p = W.paper_cdr_adi(False, 0.1, n, 2000)
    g = Grid(p, prec=args.prec)
    info = g.info()
    P, m, K = info["n_patch"], info["m_xi"], info["k_micro"]
    pts = P * m * m
    n_macro = 20
    dtm = info["dt_macro_suggested"]
    es = 4 if args.prec == "fp32" else 8
    U0 = g.init_field()
    U = U0.clone()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def run(grid, steps, warm):
        for _ in range(warm):
            U.copy_(U0)
            grid.step(U, 0.0, dtm, n_macro)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        l0 = grid.launches()
        for s in range(steps):
            U.copy_(U0)
            flush.fill_(float(s))
            ev[s][0].record(stream)
            grid.step(U, 0.0, dtm, n_macro)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev), grid.launches() - l0

    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ms, launches = run(g, args.steps, args.warmup)
    clocks = sampler.stop()
    U_adi = U.clone()
    value = pts * K * n_macro * args.steps / (ms / 1e3)
    # forward-Euler bursts of the same length tau
    probe = Grid(dict(p, micro="fe", dt_micro=None, k_micro=1, cfl_micro=1.0), prec=args.prec)
    k_fe = int(math.ceil(info["tau"] / probe.info()["dt_micro"]))
    del probe
    gf = Grid(dict(p, micro="fe", dt_micro=info["tau"] / k_fe, k_micro=k_fe), prec=args.prec)
    fe_steps = max(1, min(3, args.steps))
    ms_fe, _ = run(gf, fe_steps, 1)
    diff = (torch.linalg.norm(U - U_adi) / torch.linalg.norm(U)).item()
    del gf
    # end to end through the public API: host field in, host field out, every step
    Uh = U0.cpu().pin_memory()
    Uo = torch.empty_like(Uh).pin_memory()
    e2e_steps = max(1, args.steps // 2)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        U.copy_(Uh, non_blocking=True)
        g.step(U, 0.0, dtm, n_macro)
        Uo.copy_(U, non_blocking=True)
    torch.cuda.synchronize()
    e2e = pts * K * n_macro * e2e_steps / (time.perf_counter() - t)
    nbytes = U0.numel() * 8
    pk = peaks()
    kern_s = ms / 1e3 / (args.steps * n_macro)
    # per micro point: the forcing basis of the burst record (12 values) once,
    # the eta-line and xi-line records (2 x 8 values) in every ADI step; per
    # patch the macro value out (the 3 x 3 stencil reads hit L2)
    bytes_launch = pts * (12 * es + 16 * es * K) + P * 16
    achieved = bytes_launch / kern_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "Section 4.1.1 (lambda = 0.1) at the paper's patch settings on a %dx%d macro grid: "
                               "%d patches x %dx%d micro points, ADI bursts of %d steps (tau = %.3g), "
                               "%d macro steps per step" % (n, n, P, m, m, K, info["tau"], n_macro),
                   "point_updates_per_step": pts * K * n_macro,
                   "l2": "flushed between timed steps (512 MB write)"},
        "macro_steps_per_s": n_macro * args.steps / (ms / 1e3),
        "forward_euler_same_tau": {"k_micro": k_fe, "ms_per_macro_step": ms_fe / (fe_steps * n_macro),
                                   "adi_speedup": (ms_fe / fe_steps) / (ms / args.steps),
                                   "rel_l2_adi_vs_fe_after_20_steps": diff},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": None,
                     "kernel": "patch_adi_kernel<11,-,tsrc,%s,fused> (one macro step per launch)"
                               % ("float" if es == 4 else "double"),
                     "bytes_per_launch": bytes_launch, "kernel_ms_per_macro_step": 1e3 * kern_s,
                     "peak_source": "%s hbm_gbs" % pk["source"]},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        import oracle
        o = oracle.Oracle(p)
        Uc = U0.cpu().numpy()
        sel = np.random.default_rng(0).choice(o.n_patch, size=min(2000, o.n_patch), replace=False)
        t = time.perf_counter()
        reps = 0
        while time.perf_counter() - t < 10.0:
            o.patch_dU(Uc, 0.0, sel)
            reps += 1
        el = time.perf_counter() - t
        line["cpu_baseline"] = {"value": reps * len(sel) * m * m * K / el, "unit": UNIT,
                                "cores": oracle.num_threads(),
                                "kind": "oracle",
                                "sample": "ADI bursts of %d random patches, %d repetitions (%.1f s)"
                                          % (len(sel), reps, el)}
    print(json.dumps(line), flush=True)
    return 0


def run_refresh(args):
    """Edge-data refresh (Q > 1) on the 512x2048-node annulus (84.6 M micro
    points, K = 20, FP32 bursts): pd_step over 2 macro steps per bench step for
    Q = 2, 4, 10 (separate passes with refreshes) beside Q = 1 (fixed edge data,
    the fused path), L2 flushed between bench steps.  Roofline of the refresh
    path: its algorithmic HBM bytes per macro step against the copy bandwidth."""
    import torch

    from paper_2405_08764_gb300 import workloads as W
    from paper_2405_08764_gb300.api import Grid

    torch.cuda.set_device(0)
    n_r, n_theta = (int(v) for v in args.c5_grid.split("x"))
    base = W.c5_surrogate_field(n_r=n_r, n_theta=n_theta)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    n_macro = 2
    es = 4
    pk = peaks()
    res = {}
    sampler = ClockSampler(0)
    sampler.start()
    for Q in (1, 2, 4, 10):
        g = Grid(dict(base, q_refresh=Q), prec="fp32")
        info = g.info()
        P, m, K = info["n_patch"], info["m_xi"], info["k_micro"]
        pts = P * m * m
        dtm = info["dt_macro_suggested"]
        U0 = g.init_field()
        U = U0.clone()
        for _ in range(args.warmup):
            U.copy_(U0)
            g.step(U, 0.0, dtm, n_macro)
        torch.cuda.synchronize()
        ms = 0.0
        l0 = g.launches()
        for s in range(args.steps):
            U.copy_(U0)
            flush.fill_(float(s))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.step(U, 0.0, dtm, n_macro)
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        ms_macro = ms / (args.steps * n_macro)
        r = {"ms_per_macro_step": ms_macro, "exec_path": info["exec_path"],
             "point_updates_per_s": pts * K / (ms_macro / 1e3),
             "launches_per_macro_step": (g.launches() - l0) / (args.steps * n_macro)}
        if Q > 1:
            # lift (record in; u0, r, w out), Q bursts (w, r, 64 B record in; w out), Q restrictions
            # (w in), Q - 1 refreshes (edge points: record in, r in and out), projection
            edge_pts = P * 4 * (m - 1)
            nbytes = (pts * (32 + 8 + 2 * es) + P * (4 * (m + 2) * 8 + 8)
                      + Q * pts * (3 * es + 64) + Q * (pts * es + P * 16)
                      + (Q - 1) * (edge_pts * (32 + 2 * es) + 3 * P * 8) + P * 24)
            r["bytes_per_macro_step"] = nbytes
            r["GB_per_s"] = nbytes / (ms_macro / 1e3) / 1e9
            r["frac_hbm"] = r["GB_per_s"] / pk["hbm_gbs"]
        res["Q=%d" % Q] = r
        del g
    clocks = sampler.stop()
    q4 = res["Q=4"]
    line = {
        "metric": "edge-refresh path: point-updates/s and achieved HBM GB/s per Q", "value": q4["point_updates_per_s"],
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "annulus %dx%d macro nodes, %dx%d micro, K=%d, %d macro steps per step, Q in 1,2,4,10"
                               % (n_r + 1, n_theta, m, m, K, n_macro),
                   "l2": "flushed between timed steps (512 MB write)"},
        "roofline": {"bound": "hbm", "achieved": q4["GB_per_s"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": q4["frac_hbm"], "traffic": None, "kernel": "refresh path at Q = 4 (all its passes)",
                     "peak_source": "%s hbm_gbs" % pk["source"]},
        "per_q": res, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="c4: leave out the FP64 batch and the 65x65 problem from the line")
    ap.add_argument("--workload", default="c4", choices=["c4", "c2", "c5", "passes", "adi", "refresh"],
                    help="c4: the 4096-instance batch (default); c2: the 65x65 heterogeneous problem alone; "
                         "c5: the surrogate against the plain scheme on the 512x2048 annulus; "
                         "passes: the separate C-ABI passes on that annulus; "
                         "adi: ADI bursts at the paper's Section 4.1 patch settings; "
                         "refresh: edge-data refresh Q = 1, 2, 4, 10 on the annulus")
    ap.add_argument("--macro", type=int, default=C4_MACRO, help="c4: macro steps per bench step")
    ap.add_argument("--adi-n", type=int, default=400, help="adi: macro intervals per side")
    ap.add_argument("--epochs", type=int, default=80, help="c5: training epochs")
    ap.add_argument("--c5-grid", default="511x2048", help="c5: radial intervals x angular nodes")
    ap.add_argument("--batch", type=int, default=2048, help="c5: training minibatch")
    ap.add_argument("--instances", type=int, default=N_INST)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "c2":
        return run_c2(args)
    if args.workload == "c5":
        return run_surrogate(args)
    if args.workload == "passes":
        return run_passes(args)
    if args.workload == "adi":
        return run_adi(args)
    if args.workload == "refresh":
        return run_refresh(args)
    return run_batch(args)


if __name__ == "__main__":
    sys.exit(main())
