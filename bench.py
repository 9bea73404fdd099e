#!/usr/bin/env python
"""Benchmark of the GPU random walk: particle histories per second and figure of merit.

Workload (default): the largest single-GPU configuration, a 17 x 17 lattice of pins (r 0.54 cm,
pitch 1.26 cm) in a reflective box, 7 groups, three seeded materials with secondary production
scaled to spectral radius 0.9, uniform volumetric pulse source, a 34 x 34 x 7 x 50 space-group-time
mesh tally (404,600 bins), 1e8 histories per step, FP32 tracking, int64 fixed-point tallies, 32
statistical batches.  One step = one mc_run over all histories: source sampling, the persistent
event loop (flight, track-length scoring, collision, surface, secondaries), and the batch
statistics.  Inputs are seeded synthetic cross sections.  `--workload config2` (7-group infinite
medium pulse, 1e7 histories) and the others listed in `workload()` print the same line.

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


KERNEL_SOURCES = {
    "k_transport": ["mc_transport.cuh", "mc_transport.cu", "mc_transport_seg.cu", "mc_transport_range.cu",
                    "mc_events.cuh", "mc_device.cuh", "mc_internal.h"],
    "k_transport_batch": ["mc_batch.cu", "mc_events.cuh", "mc_device.cuh", "mc_internal.h"],
}


def source_digest(kernel):
    """Digest of the sources a kernel is compiled from (comments removed) and of the ABI header:
    identifies the kernel build an ncu summary was taken on."""
    import hashlib
    import re
    h = hashlib.sha256()
    files = [os.path.join(ROOT, "paper_2305_07636_gb300", "csrc", f) for f in KERNEL_SOURCES[kernel]]
    for f in files + [os.path.join(ROOT, "include", "mc.h")]:
        with open(f) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(os.path.basename(f).encode() + b"\0" + text.encode())
    return h.hexdigest()[:16]


def profiled_value(summary, kernel, key):
    """A number recorded in a committed ncu summary under profiles/ (`key: value`), or None when the
    summary was taken on other kernel sources than these."""
    import re
    try:
        with open(os.path.join(ROOT, "profiles", summary)) as f:
            text = f.read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9.eE+]+)", text)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    if m and d and d.group(1) == source_digest(kernel):
        return float(m.group(1))
    return None


def traffic_per_launch(workload, flights):
    """DRAM bytes (read + write) of one transport launch of this run: the committed ncu summary's
    DRAM bytes per flight (captured on a smaller case of the same workload, whose traffic grows in
    proportion to the flights) times this launch's flights; None when the summary was taken on
    other kernel sources than these."""
    per_flight = profiled_value(f"k_transport_{workload}.md", "k_transport", "traffic_bytes_per_flight")
    return None if per_flight is None else per_flight * flights


def workload(name):
    from paper_2305_07636_gb300 import problems as P
    if name == "config2":
        return P.config2(), 10_000_000, "config2: 7-group infinite medium pulse, 1e7 histories"
    if name == "config2x":
        return P.config2_crossing(), 10_000_000, ("config2x: 7-group infinite medium pulse, 1e7 histories, "
                                                  "track-length and time-crossing tallies")
    if name == "config1":
        return P.config1(), 10_000_000, "config1: 1-group slab, 1e7 histories"
    if name == "config3":
        return P.config3(), 100_000_000, ("config3: 17x17 pin lattice (r 0.54, pitch 1.26 cm, reflective), 7 groups, "
                                          "3 seeded materials, spectral radius 0.9, mesh 34x34x7x50, 1e8 histories")
    if name == "config4":
        return P.config4(), 1_000_000, ("config4: 200 cm stack of 40 layers (4 seeded materials, Sigma_t "
                                        "0.5-3, c 0.3-0.95), 7 groups, cosine surface source at x=0, "
                                        "detector 198-200 cm; learned weight windows")
    if name == "pc":
        return P.azurv1(), 10_000_000, ("pc: supercritical AZURV1 (c = 1.1, 20 mean free times), population control "
                                        "by splitting-roulette at a census every 2 mean free times, 1e7 histories")
    if name == "eigen":
        return P.pin_cell(), 1_000_000, ("eigen: k-eigenvalue power iteration of a 7-group pin cell (pin r 0.54 cm, "
                                        "pitch 1.26 cm, reflective; seeded cross sections), 50 inactive + 100 "
                                        "active cycles of 1e6 histories")
    if name == "config5":
        probs, nh = P.config5()
        return (probs, nh), sum(nh), (f"config5: {len(probs)} independent problems (1D/2D slab, "
                                      f"pin lattice; 1-7 groups), {sum(nh)} histories in all, "
                                      f"{min(nh)}-{max(nh)} per problem")
    raise SystemExit(f"unknown workload {name}")


def oracle_batch_fraction(probs, nh, threads, target_s, seed):
    """Fraction of every problem's histories that the oracle runs in about target_s seconds."""
    import oracle
    frac = 1e-3
    t0 = time.perf_counter()
    for i, (q, n) in enumerate(zip(probs, nh)):
        oracle.run(q, max(32, int(n * frac)), seed=seed + i, threads=threads)
    dt = time.perf_counter() - t0
    return min(1.0, frac * target_s / max(dt, 1e-3))


def oracle_batch_sample(probs, nh, threads, frac, seed):
    """The oracle over every problem of a batch with its history count scaled by frac;
    returns (histories, seconds)."""
    import oracle
    t0 = time.perf_counter()
    n1 = 0
    for i, (q, n) in enumerate(zip(probs, nh)):
        m = max(32, int(n * frac))
        oracle.run(q, m, seed=seed + i, threads=threads)
        n1 += m
    return n1, time.perf_counter() - t0


def issue_roofline(workload, n, flights, kernel_ms, clk):
    """Instruction issue of the transport kernel against the issue peak of 152 SMs x 4 warp schedulers
    x the SM clock seen during the timed region (one warp instruction per scheduler per clock): the
    ceiling this latency-bound kernel actually meets.  The warp instructions per flight come from the
    committed ncu summary of the same kernel sources (None when they changed)."""
    per_flight = profiled_value(f"k_transport_{workload}.md", "k_transport", "warp_instructions_per_flight")
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    if per_flight is None:
        return None
    achieved = per_flight * flights / (kernel_ms / 1000.0)
    peak = 152 * 4 * mhz * 1e6
    return {"bound": "issue", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G warp instructions/s",
            "frac": achieved / peak, "warp_instructions_per_flight": per_flight,
            "peak_kind": "152 SMs x 4 schedulers x SM clock sampled during the timed region"}


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
    if args.workload == "config5":
        return run_reference_batch(args, prob, n_full, desc, threads)
    probe = 20000
    t0 = time.perf_counter()
    oracle.run(prob, probe, seed=1, threads=threads)
    per = (time.perf_counter() - t0) / probe
    # each step is a bounded sample: the whole --steps K run stays within about 2.5 minutes
    step_s = min(args.ref_step_seconds, 150.0 / max(1, args.steps))
    n = int(max(probe, min(n_full, step_s / per)))
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


def run_reference_batch(args, batch, n_full, desc, threads):
    probs, nh = batch
    frac = oracle_batch_fraction(probs, nh, threads, min(args.ref_step_seconds, 150.0 / max(1, args.steps)), 7)
    hist, secs = 0, 0.0
    for k in range(args.steps):
        n, dt = oracle_batch_sample(probs, nh, threads, frac, 100 + 1000 * k)
        hist += n
        secs += dt
    value = hist / secs
    sample = (f"every problem of the batch with its histories scaled by {frac:.2e}, FP64 C++ oracle, "
              f"{threads} threads, problems one after another")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * secs / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample_fraction": frac},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def pct(a, q):
    return float(np.percentile(np.asarray(a, dtype=np.float64), q))


def bench_batch(args, torch, mc, batch, n_total, desc, world, local):
    """One step = one batched launch (mc_run_batch) of all problems, after the autotuner has
    chosen the configuration (untimed).  The sequential comparison runs the same problems, same
    seeds, one mc_run after another on the same stream."""
    probs, nh = batch
    ps = [mc.Problem(q) for q in probs]
    hs = [p.h for p in ps]
    stream = torch.cuda.current_stream()
    seed = 5
    extra = {k: int(v) for k, v in (o.split("=", 1) for o in args.opt)}
    bopts = mc.run_opts(**extra) if extra else None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    tuned, tune_ms = mc.batch_tune(hs, nh, seed, bopts, stream)
    tune_s = time.perf_counter() - t0
    for w in range(args.warmup):
        flush.zero_()
        mc.run_batch(hs, nh, seed + w, bopts, stream)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for k in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        ev_s[k].record(stream)
        mc.run_batch(hs, nh, seed + 100 + k, bopts, stream)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    for p in ps:
        p.wait()
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    ms_per_step = sum(step_ms) / len(step_ms)
    value = n_total / (ms_per_step / 1000.0)
    # per-problem completion times since the launch started (device clock), untimed extra step
    wall = mc.run_batch(hs, nh, seed + 100, bopts, stream, wall=True)
    cs = [p.counters() for p in ps]
    flights = sum(c["flight"] for c in cs)
    scores = sum(c["scores"] for c in cs)
    kernel_ms = 1000.0 * float(wall.max())

    # sequential: the same problems and seeds, one mc_run each, shortest first
    order = np.argsort(nh, kind="stable")
    seq_steps = max(1, min(args.steps, 3))
    seq_ms, seq_done = [], None
    for k in range(seq_steps + 1):
        flush.zero_()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(ps) + 1)]
        evs[0].record(stream)
        for j, i in enumerate(order):
            mc.run(ps[i].h, nh[i], seed + 100 + i, None, stream)
            evs[j + 1].record(stream)
        torch.cuda.synchronize()
        if k == 0:
            continue  # warm-up
        done = np.array([evs[0].elapsed_time(evs[j + 1]) for j in range(len(ps))]) / 1000.0
        seq_ms.append(1000.0 * done[-1])
        seq_done = np.empty(len(ps))
        seq_done[order] = done
    seq_value = n_total / (statistics.mean(seq_ms) / 1000.0)

    peak, peak_kind = peaks()
    algo_bytes = flights * BYTES_PER_FLIGHT
    achieved = algo_bytes / (kernel_ms / 1000.0) / 1e9
    atom_peak = mc.atomic_peak(1 << 24)

    # end to end through the public API with host buffers: create every problem (tables to the
    # device), one batched launch, read every tally and leakage back, destroy
    e2e_times, h2d, d2h = [], 0, 0
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qs = [mc.Problem(q) for q in probs]
        mc.run_batch([q.h for q in qs], nh, seed + 500 + k, None, stream)
        h2d, d2h = 0, 0
        for q, pr in zip(qs, probs):
            for t in range(len(pr["tallies"])):
                m, e = q.tally(t)
                d2h += 3 * 8 * m.size
            lm, ls = q.leakage()
            d2h += 3 * 8 * lm.size
            h2d += q.table_bytes()
        for q in qs:
            q.close()
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = n_total / statistics.median(e2e_times) if e2e_times else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "histories_per_step": n_total, "tracking": "fp32",
                   "tally": "int64 fixed point 2^-32", "batches": 32,
                   "launch": "mc_run_batch (one persistent launch replayed from a CUDA graph)",
                   "tuned": {"block_size": tuned.block_size, "blocks_per_sm": tuned.blocks_per_sm,
                             "batch_unit": tuned.batch_unit},
                   "l2": "flushed (256 MB write) before every timed step"},
        "batch": {"problems": len(ps), "autotune_s": tune_s, "tuned_launch_ms": tune_ms,
                  "per_problem_wall_s": {"p50": pct(wall, 50), "p99": pct(wall, 99),
                                         "max": float(wall.max())},
                  "sequential": {"value": seq_value, "ms_per_step": statistics.mean(seq_ms),
                                 "per_problem_wall_s": {"p50": pct(seq_done, 50),
                                                        "p99": pct(seq_done, 99),
                                                        "max": float(seq_done.max())},
                                 "launch": "one mc_run per problem, shortest first, same stream"},
                  "speedup_vs_sequential": value / seq_value},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_value("k_transport_batch_config5.md", "k_transport_batch", "traffic_bytes_per_launch"),
                     "kernel": "k_transport_batch<float>", "kernel_ms": kernel_ms,
                     "algorithmic_bytes": algo_bytes, "peak_kind": peak_kind,
                     "l2_atomic": {"achieved": scores / (kernel_ms / 1000.0) / 1e9,
                                   "peak": atom_peak / 1e9, "unit": "G atomics/s",
                                   "frac": scores / (kernel_ms / 1000.0) / atom_peak,
                                   "peak_kind": "measured live (mc_atomic_peak, random 64-bit adds)"}},
        "counters": {"flight": flights, "scores": scores},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "step_ms": [round(x, 4) for x in step_ms],
    }
    if not args.no_cpu_baseline and world == 1:
        frac = oracle_batch_fraction(probs, nh, os.cpu_count() or 1, 10.0, 9)
        n, dt = oracle_batch_sample(probs, nh, os.cpu_count() or 1, frac, 9000)
        line["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": os.cpu_count() or 1,
                                "kind": "oracle",
                                "sample": f"every problem with its histories scaled by {frac:.2e}"}
    print(json.dumps(line), flush=True)
    for p in ps:
        p.close()


def detector_stats(p, nb=32):
    """Detector total (tally 0, all bins) per batch: mean and standard error per source history."""
    b = p.tally_batches(0).reshape(nb, -1).sum(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(len(b))), int(np.count_nonzero(b))


def learn_windows(mc, P, p, prob, rounds, n0, n_round, seed, extrap=(1.0, 80.0), epochs=3000):
    """Analog run, then `rounds` refinement rounds: learn the windows from the last run's
    training tally (tally 1), run with them.  Returns the network and a per-round record."""
    p.run(n0, seed, tally_mode="fp64")
    p.wait()
    net = mc.Mlp(P.mlp_init(seed=4))
    xs = np.asarray(prob["tallies"][1]["x"])
    log = []
    for r in range(rounds):
        t0 = time.perf_counter()
        info = mc.ww_learn(p.h, net, 1, epochs, 3e-3, *extrap)
        learn_s = time.perf_counter() - t0
        p.run(n_round, seed + 1 + r, tally_mode="fp64", ww_enable=1, bank_capacity=1 << 25)
        p.wait()
        m, s, _ = detector_stats(p)
        mean, err = p.tally(1)
        ok = ((err < 0.5 * np.abs(mean)) & (mean > 0)).reshape(len(xs) - 1, -1)
        depth = float(xs[1:][ok.any(axis=1)].max()) if ok.any() else 0.0
        log.append({"round": r + 1, "resolved_points": info["points"],
                    "extrapolated_points": info["extrapolated"], "loss": info["loss"],
                    "learn_s": learn_s, "run_ms": p.timing()[0], "detector": m,
                    "detector_rel": s / m if m > 0 else None, "resolved_depth_cm": depth})
    return net, log


def timed_fom(torch, mc, p, n, seed, stream, **opts):
    """One run timed with CUDA events: detector mean, relative error, seconds, FOM."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o = mc.run_opts(tally_mode="fp64", **opts)
    e0.record(stream)
    mc.run(p.h, n, seed, o, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    p.wait()
    t = e0.elapsed_time(e1) / 1000.0
    m, s, nz = detector_stats(p)
    rel = s / m if m > 0 else None
    return {"histories": n, "seconds": t, "detector": m, "std_err": s, "rel_err": rel,
            "batches_scoring": nz, "fom": 1.0 / (rel * rel * t) if rel else 0.0,
            "histories_per_s": n / t}


EIGEN_CYCLES = (50, 100)  # inactive, active: the paper's C5G7 k-eigenvalue run


def bench_eigen(args, torch, mc, prob, n, desc):
    """One step = one whole power iteration (50 inactive + 100 active cycles of n histories, as the
    paper's k-eigenvalue run) through mc_run_eigen, timed with CUDA events around the call (it
    synchronises once per cycle to read k).  value = histories of all cycles / time."""
    ni, na = EIGEN_CYCLES
    p = mc.Problem(prob)
    stream = torch.cuda.current_stream()
    extra = {k: int(v) for k, v in (o.split("=", 1) for o in args.opt)}
    opts = mc.run_opts(**extra) if extra else None
    for w in range(args.warmup):
        mc.run_eigen(p.h, n, 2, 2, 1000 + w, opts, stream)
    clocks = Clocks(0)
    times, ks = [], []
    for k in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        kc, sites, km, ke = mc.run_eigen(p.h, n, ni, na, 7 + k, opts, stream)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b) / 1000.0)
        ks.append((km, ke))
    clk = clocks.stop()
    c = p.counters()
    tr_ms, st_ms = p.timing()
    t = sum(times) / len(times)
    hist = n * (ni + na)
    value = hist / t
    km, ke = ks[-1]
    fom = 1.0 / ((ke / km) ** 2 * t)
    peak, peak_kind = peaks()
    achieved = c["flight"] * BYTES_PER_FLIGHT / t / 1e9
    # end to end: create the problem (tables host->device), iterate, read the tallies back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q = mc.Problem(prob)
    mc.run_eigen(q.h, n, ni, na, 99, opts, stream)
    mean, err = q.tally(0)
    h2d = q.table_bytes()
    q.close()
    e2e = hist / (time.perf_counter() - t0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "histories_per_cycle": n, "cycles": {"inactive": ni, "active": na},
                   "tracking": "fp32", "tally": "int64 fixed point 2^-32", "run_opts": extra},
        "k": {"mean": km, "std_err": ke, "fom_1_per_s": fom,
              "paper_context": "MC/DC 2563.8 s (incl. ~63 s JIT) and Shift 1020.7 s for 1e5 x 150 cycles of the "
                               "C5G7 UO2 pin cell on LLNL Lassen (IBM POWER9), i.e. ~6.0e3 and ~1.47e4 "
                               "source particles/s"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_transport<float>", "peak_kind": peak_kind,
                     "note": "algorithmic bytes over the whole iteration time (per-cycle syncs included)"},
        "counters": {k: c[k] for k in ("flight", "collision", "production", "secondary")},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 3 * 8 * mean.size},
        "gpu_launches": (ni + na) * 5 + 2,
        "clocks": clk,
        "step_s": [round(x, 4) for x in times],
    }
    if not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        ns = 20000
        t0 = time.perf_counter()
        oracle.run_eigen(prob, ns, 5, 10, seed=5, threads=threads)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns * 15 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{ns} histories x 15 cycles, FP64 C++ oracle"}
    print(json.dumps(line), flush=True)
    p.close()


def time_learning_kernels(torch, mc, P, n=700, epochs=3000, reps=5):
    """CUDA-event times of the importance network's kernels on n training points (the 200 cm stack's
    learning rounds train on about 700): one forward pass, one loss-and-gradient pass, and full-batch
    Adam (one launch for all epochs), per call and per epoch."""
    rng = np.random.default_rng(1)
    x = torch.tensor(P.bf16_round(rng.uniform(-1, 1, (n, 5))), dtype=torch.float32, device="cuda")
    tgt = torch.tensor(rng.normal(0, 1, n), dtype=torch.float32, device="cuda")
    wt = torch.ones(n, dtype=torch.float32, device="cuda")
    y = torch.zeros(n, device="cuda")
    net = mc.Mlp(P.mlp_init(seed=4))
    g = torch.zeros(net.n_params, device="cuda")
    loss = torch.zeros(1, device="cuda")

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    fwd = timed(lambda: net.forward(x.data_ptr(), y.data_ptr(), n), 20 * reps)
    grad = timed(lambda: net.loss_grad(x.data_ptr(), tgt.data_ptr(), wt.data_ptr(), n, g.data_ptr(),
                                       loss.data_ptr()), 20 * reps)
    train = timed(lambda: net.train(x.data_ptr(), tgt.data_ptr(), wt.data_ptr(), n, epochs, 3e-3, loss.data_ptr()),
                  reps)
    net.close()
    flops_fwd = 2.0 * (5 * 64 + 2 * 64 * 64 + 64) * n
    return {"points": n, "forward_ms": fwd, "loss_grad_ms": grad, "train_ms": train, "epochs": epochs,
            "train_ms_per_epoch": train / epochs, "forward_tflops": flops_fwd / (fwd * 1e-3) / 1e12,
            "note": "one cooperative launch trains for all epochs on a grid of CTAs (a warp per 16-sample "
                    "tile, two grid barriers per epoch); the network is 8,769 parameters"}


def bench_learned_ww(args, torch, mc):
    """Learned weight windows on the 200 cm stack: 5 refinement rounds from an analog start,
    then a measurement run with the final windows; analog and an exponential (non-learned) window
    table on the same GPU for comparison; the same pipeline on a 10 cm stack that analog can
    score, for the analog FOM ratio and the bias check."""
    from paper_2305_07636_gb300 import problems as P
    stream = torch.cuda.current_stream()
    prob = P.config4()
    p = mc.Problem(prob)
    t0 = time.perf_counter()
    net, rounds = learn_windows(mc, P, p, prob, 5, 4_000_000, 1_000_000, 4)
    learn_total = time.perf_counter() - t0
    for w in range(args.warmup):
        mc.run(p.h, 200_000, 50 + w, mc.run_opts(tally_mode="fp64", ww_enable=1, bank_capacity=1 << 25), stream)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    steps = [timed_fom(torch, mc, p, 2_000_000, 100 + k, stream, ww_enable=1, bank_capacity=1 << 25)
             for k in range(args.steps)]
    clk = clocks.stop()
    sec = sum(x["seconds"] for x in steps)
    mean = float(np.mean([x["detector"] for x in steps]))
    # the steps are independent: pool them (variance of the mean of K estimates)
    se = math.sqrt(sum(x["std_err"] ** 2 for x in steps)) / len(steps)
    rel = se / mean if mean > 0 else None
    learned = {"histories": sum(x["histories"] for x in steps), "seconds": sec, "detector": mean,
               "std_err": se, "rel_err": rel, "fom": 1.0 / (rel * rel * sec) if rel else 0.0,
               "seconds_to_5pct": sec * (rel / 0.05) ** 2 if rel else None}
    c = p.counters()
    # analog on the same problem: no history reaches the detector
    n_an = 100_000_000
    analog = timed_fom(torch, mc, p, n_an, 7, stream)
    analog["upper_bound_note"] = ("no score in %d histories: fewer than 3 in %d histories reach the "
                                  "detector at 95%% confidence" % (n_an, n_an))
    # non-learned windows: one exponential in x for all groups, decay fitted to the analog flux
    p.run(4_000_000, 4, tally_mode="fp64")
    fm, fe = p.tally(1)
    xs = np.asarray(prob["tallies"][1]["x"])
    tot = fm.reshape(len(xs) - 1, -1).sum(axis=1)
    ok = tot > 0
    xc = 0.5 * (xs[:-1] + xs[1:])
    decay = float(-np.polyfit(xc[ok], np.log(tot[ok]), 1)[0])
    p.set_weight_windows(P.exponential_ww(prob, decay))
    try:
        expo = timed_fom(torch, mc, p, 2_000_000, 9, stream, ww_enable=1, bank_capacity=1 << 25)
    except mc.McError as e:
        expo = {"failed": str(e)}
    expo["decay_per_cm"] = decay
    p.close()
    # thin variant: analog scores, so analog FOM and the bias check are measured
    thin = P.slab_stack(thickness=10.0, n_layers=5, detector=2.0, ww_bin=1.0, name="thin")
    q = mc.Problem(thin)
    an = timed_fom(torch, mc, q, 100_000_000, 11, stream)
    net2, rounds2 = learn_windows(mc, P, q, thin, 5, 4_000_000, 1_000_000, 12)
    lw = timed_fom(torch, mc, q, 2_000_000, 13, stream, ww_enable=1, bank_capacity=1 << 25)
    z = (lw["detector"] - an["detector"]) / math.hypot(lw["std_err"], an["std_err"])
    q.close()
    net.close()
    net2.close()
    value = learned["histories"] / sec
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * sec / len(steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload("config4")[2], "histories_per_step": 2_000_000,
                   "tracking": "fp32", "tally": "fp64 atomics", "batches": 32,
                   "windows": "MLP 5-64-64-64-1 (BF16 tensor cores, FP32 accumulate), 5 rounds "
                              "from a 4e6-history analog run, 1e6 histories per round, "
                              "extrapolation slope 1.0 over 80 e-folds",
                   "l2": "inputs (particle banks) larger than L2 between steps"},
        "fom": {"learned": learned, "analog": analog, "exponential_ww": expo,
                "thin_10cm": {"analog": an, "learned": lw, "fom_ratio": lw["fom"] / an["fom"] if an["fom"] else None,
                              "z_learned_vs_analog": z, "rounds": rounds2},
                "unit": "1/s", "tally": "detector flux, last 2 cm, all groups"},
        "rounds": rounds, "learning_s": learn_total,
        "learning_kernels": time_learning_kernels(torch, mc, P),
        "counters": {k: c[k] for k in ("flight", "ww_split", "ww_kill", "scores")},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "step_ms": [round(1000 * x["seconds"], 3) for x in steps],
    }
    print(json.dumps(line), flush=True)


def probes(torch, mc):
    """The measured figures the design rests on (not a benchmark step): instruction throughput per SM
    clock (mc_op_rates) and 64-bit L2 atomic rates over spans of slots from one address to a
    footprint far beyond L2 (mc_atomic_peak)."""
    spans = [1, 700, 22_400, 360_000, 1_000_000, 13_000_000, 100_000_000]
    line = {"probes": "instruction and atomic rates", "op_rates_per_clk_per_sm": mc.op_rates(),
            "l2_atomics_per_s": {str(sp): mc.atomic_peak(sp) for sp in spans},
            "device": torch.cuda.get_device_name(0)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)  # ~4 s timed on the default workload
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config3")
    ap.add_argument("--histories", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--algorithm", default="auto", choices=["auto", "event", "history"],
                    help="auto: the autotuner picks event- or history-based (identical results)")
    ap.add_argument("--no-flush", action="store_true", help="skip the L2 flush between steps")
    ap.add_argument("--no-tune", action="store_true", help="skip the kernel autotuner (library defaults)")
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
    if args.workload == "probes":
        return probes(torch, mc)
    prob, n, desc = workload(args.workload)
    if args.workload == "config4":
        if world > 1:
            raise SystemExit("the learned-window workload runs on one GPU")
        return bench_learned_ww(args, torch, mc)
    if args.workload == "config5":
        if world > 1:
            raise SystemExit("the batched workload runs on one GPU")
        return bench_batch(args, torch, mc, prob, n, desc, world, local)
    if args.workload == "eigen":
        if world > 1:
            raise SystemExit("the k-eigenvalue workload runs on one GPU")
        return bench_eigen(args, torch, mc, prob, args.histories or n, desc)
    if args.histories:
        n = args.histories
    seed = 2
    p = mc.Problem(prob)
    extra = {k: int(v) for k, v in (o.split("=", 1) for o in args.opt)}
    census = {"census_times": np.arange(2.0, 20.0, 2.0)} if args.workload == "pc" else {}
    opts = mc.run_opts(first_history=rank * n, algorithm=args.algorithm, **extra, **census)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    tuned = None
    if not extra and not args.no_tune:
        # the kernel configuration for this problem, picked by the library's autotuner (untimed)
        t_opts, tune_ms = mc.run_tune(p.h, n, seed, opts, stream)
        tuned = {"block_size": t_opts.block_size, "blocks_per_sm": t_opts.blocks_per_sm,
                 "algorithm": ["event", "history"][t_opts.algorithm],
                 "drain_threshold": t_opts.drain_threshold or "default", "candidate_ms": tune_ms}
    algorithm = tuned["algorithm"] if tuned and args.algorithm == "auto" else (
        "event" if args.algorithm == "auto" else args.algorithm)
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
    combined = None
    if dist is not None:
        t = torch.tensor([t_dev], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())
        # the one exchange step of sharded histories (after the timed region): every rank's exact
        # int64 tally sums of its last run, added by one all-reduce into the sums of the union of
        # the ranks' history ranges
        sums, bits = mc.tally_sums(p.h, 0)
        ts = torch.from_numpy(sums.ravel()).to("cuda")
        dist.all_reduce(ts)
        tot = ts.cpu().numpy()
        combined = {"bins": int(tot.size), "fixed_bits": bits, "ranks": world,
                    "histories": world * n, "total_flux": float(tot.sum()) / 2.0 ** bits / (world * n)}
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
    # tally scoring against the L2 atomic roofline, measured live on the run's own tally footprint
    # (stripes x batches x row elements, as the library laid it out)
    stripes, n_batches, row = mc.tally_layout(p.h)
    footprint = stripes * n_batches * row
    atom_peak = mc.atomic_peak(min(1 << 27, max(1, footprint)))
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
                   "algorithm": algorithm, "run_opts": extra, "tuned": tuned,
                   "tally": "int64 fixed point 2^-32", "batches": opts.n_batches,
                   "l2": "flushed (256 MB write) before every timed step"},
        "fom": {"value": fom, "unit": "1/s", "tally": "total flux (all groups and time bins)",
                "rel_err_per_step": rel, "seconds_to_5pct": t_5pct},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic_per_launch(args.workload, c["flight"]),
                     "kernel": "k_transport<float>", "kernel_ms": tr_ms,
                     "algorithmic_bytes": algo_bytes, "peak_kind": peak_kind,
                     "l2_atomic": {"achieved": atom_rate / 1e9, "peak": atom_peak / 1e9,
                                   "unit": "G atomics/s", "frac": atom_rate / atom_peak,
                                   "scores_per_flight": c["scores"] / c["flight"],
                                   "peak_kind": "measured live (mc_atomic_peak, random 64-bit adds over the "
                                                f"run's tally footprint: {stripes} stripes x {n_batches} "
                                                f"batches x {row} elements)"},
                     "issue": issue_roofline(args.workload, n, c["flight"], tr_ms, clk)},
        "counters": {k: c[k] for k in ("flight", "collision", "surface", "census", "iterations")},
        "algorithm": algorithm,
        "trace": {"iterations": int(len(tr_t)), "history_style_iterations": int(tr_drain.sum()),
                  "ms_in_history_style_tail": drain_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": p.launches() * args.steps,  # counted by the library for the last run
        "combined_tally": combined,
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
