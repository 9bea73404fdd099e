#!/usr/bin/env python
"""Benchmark of the GPU random walk: particle histories per second and figure of merit.

Workload (default): the 7-group infinite homogeneous medium (reflective 10 cm cube, pulse in
group 1 at t = 0, 100 log-spaced time bins, census at 1e-3 s), 1e7 histories per step, FP32
tracking, int64 fixed-point tallies, 32 statistical batches.  One step = one mc_run over all
histories: source sampling, the persistent event loop (flight, track-length scoring, collision,
surface), and the batch statistics.  Inputs are seeded synthetic cross sections.

Our arm (default): times K steps with CUDA events on the launching stream after W warm-up steps;
L2 is flushed (256 MB write) before every timed step, outside the timed interval.  The `e2e`
figure times the public API with host buffers: mc_problem_create (tables host->device), mc_run,
mc_tally_get (device->host) and mc_problem_destroy, per step.
Reference arm (--impl reference): the CPU oracle (plain C++ FP64) on the host cores, on a bounded
sample of the same workload.
Multi-GPU (torchrun): every rank runs its own disjoint history range (no collective on the data
path); value = histories of all ranks / max over ranks of the device time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle histories/sec and FOM 1/(σ²T) at 5% rel. err, GPU vs CPU oracle"
UNIT = "histories/s"
BYTES_PER_FLIGHT = 136  # 64 B state read + 64 B state write + 8 B tally update per event


def workload(name):
    from paper_2305_07636_gb300 import problems as P
    if name == "config2":
        return P.config2(), 10_000_000, "config2: 7-group infinite medium pulse, 1e7 histories"
    if name == "config1":
        return P.config1(), 10_000_000, "config1: 1-group slab, 1e7 histories"
    if name == "config3":
        return P.config3(), 10_000_000, "config3: 17x17 pin lattice, 7 groups, 1e7 histories"
    raise SystemExit(f"unknown workload {name}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(prob, target_s=10.0, seed=123):
    """The oracle as it stands, on all host cores, over a sample sized to ~target_s seconds."""
    import oracle
    threads = os.cpu_count() or 1
    n = 20000
    t0 = time.perf_counter()
    oracle.run(prob, n, seed=seed, threads=threads)
    dt = time.perf_counter() - t0
    n2 = int(min(5e7, max(n, n * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.run(prob, n2, seed=seed + 1, threads=threads)
    dt2 = time.perf_counter() - t0
    return {"value": n2 / dt2, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n2} histories of the same workload, FP64, std::thread over history ranges"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    prob, n_full, desc = workload(args.workload)
    threads = os.cpu_count() or 1
    probe = 20000
    t0 = time.perf_counter()
    oracle.run(prob, probe, seed=1, threads=threads)
    per = (time.perf_counter() - t0) / probe
    n = int(max(probe, min(n_full, args.ref_step_seconds / per)))
    for w in range(args.warmup):
        oracle.run(prob, min(n, probe), seed=100 + w, threads=threads)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(prob, n, seed=1000 + k, threads=threads)
        times.append(time.perf_counter() - t0)
    value = n * len(times) / sum(times)
    sample = f"{n} of {n_full} histories per step, FP64 C++ oracle, {threads} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample_histories": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config2")
    ap.add_argument("--histories", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--algorithm", default="event", choices=["event", "history"])
    ap.add_argument("--no-flush", action="store_true", help="skip the L2 flush between steps")
    ap.add_argument("--opt", action="append", default=[],
                    help="extra mc_run_opts field as key=value (e.g. block_size=128)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2305_07636_gb300 import mc

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob, n, desc = workload(args.workload)
    if args.histories:
        n = args.histories
    seed = 2
    p = mc.Problem(prob)
    extra = {k: int(v) for k, v in (o.split("=", 1) for o in args.opt)}
    opts = mc.run_opts(first_history=rank * n, algorithm=args.algorithm, **extra)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for w in range(args.warmup):
        flush.zero_()
        mc.run(p.h, n, seed + w, opts, stream)
    mc.wait(p.h)
    barrier()
    clocks = Clocks(local)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    transport_ms = []
    wall0 = time.perf_counter()
    for k in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        ev_s[k].record(stream)
        mc.run(p.h, n, seed + 100 + k, opts, stream)
        ev_e[k].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    mc.wait(p.h)
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    t_dev = sum(step_ms) / 1000.0
    if dist is not None:
        t = torch.tensor([t_dev], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())
    value = world * n * args.steps / t_dev
    ms_per_step = 1000.0 * t_dev / args.steps

    # statistics, roofline and counters from the last timed run
    tr_ms, st_ms = p.timing()
    c = p.counters()
    tr_t, tr_w, tr_s, tr_drain = p.trace()
    drain_ms = float((tr_ms * 1e6 - tr_t[tr_drain][0]) / 1e6) if tr_drain.any() else 0.0
    per_batch = p.tally_batches(0).reshape(opts.n_batches, -1).sum(axis=1)
    total = per_batch.mean()
    rel = per_batch.std(ddof=1) / math.sqrt(len(per_batch)) / abs(total)
    fom = 1.0 / (rel * rel * (ms_per_step / 1000.0))
    t_5pct = (ms_per_step / 1000.0) * (rel / 0.05) ** 2
    peak, peak_kind = peaks()
    algo_bytes = c["flight"] * BYTES_PER_FLIGHT
    achieved = algo_bytes / (tr_ms / 1000.0) / 1e9
    # tally scoring against the L2 atomic roofline, measured live on the tally's footprint
    tally_elems = sum(int(np.prod(mc.tally_shape(p.h, t))) for t in range(len(prob["tallies"]) + 1))
    atom_peak = mc.atomic_peak(max(1, tally_elems * opts.n_batches * 16))
    atom_rate = c["scores"] / (tr_ms / 1000.0)

    # end to end through the public API with host buffers
    e2e_times = []
    h2d = d2h = 0
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q = mc.Problem(prob)
        mc.run(q.h, n, seed + 500 + k, opts, stream)
        mean, err = q.tally(0)
        lm, ls = q.leakage()
        h2d = q.table_bytes()
        q.close()
        e2e_times.append(time.perf_counter() - t0)
        d2h = 3 * 8 * (mean.size + lm.size)
    e2e_value = n / statistics.median(e2e_times) if e2e_times else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "histories_per_step": n, "tracking": "fp32",
                   "algorithm": args.algorithm, "run_opts": extra,
                   "tally": "int64 fixed point 2^-32", "batches": opts.n_batches,
                   "l2": "flushed (256 MB write) before every timed step"},
        "fom": {"value": fom, "unit": "1/s", "tally": "total flux (all groups and time bins)",
                "rel_err_per_step": rel, "seconds_to_5pct": t_5pct},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_transport<float>", "kernel_ms": tr_ms,
                     "algorithmic_bytes": algo_bytes, "peak_kind": peak_kind,
                     "l2_atomic": {"achieved": atom_rate / 1e9, "peak": atom_peak / 1e9,
                                   "unit": "G atomics/s", "frac": atom_rate / atom_peak,
                                   "scores_per_flight": c["scores"] / c["flight"],
                                   "peak_kind": "measured live (mc_atomic_peak, random 64-bit adds)"}},
        "counters": {k: c[k] for k in ("flight", "collision", "surface", "census", "iterations")},
        "algorithm": args.algorithm,
        "trace": {"iterations": int(len(tr_t)), "history_style_iterations": int(tr_drain.sum()),
                  "ms_in_history_style_tail": drain_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "wall_s": wall,
        "step_ms": [round(x, 4) for x in step_ms],
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(prob)
    if rank == 0:
        print(json.dumps(line), flush=True)
    p.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
