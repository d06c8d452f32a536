"""Benchmark: population fitness evaluation of ordered rule sets on one GB300 (or N, one per rank).

Headline workload: the ragged batched hard evaluation -- P=4096 rule sets with R~U{1..64} rules
of C~U{1..8} conditions, N=2^20 samples x F=128 float32 features, 10 classes -- evaluated through
the C ABI (rs_eval_hard) against a resident dataset. One step = one full population evaluation
(packing + validation + the evaluator kernel + exact counts). value = nominal condition-evals/s
(sum over sets and rules of the rule's condition count x N, per second), summed over ranks.

Extra legs on the same line (N = 1 only): the soft fine-tuning pass (P=1024 x R=32 x C=4,
N=262144, F=64, tau=0.1, forward + adjoint), the device-resident evolution loop, serving, the
categorical workload and the paper's plain shape. The CPU oracle is timed on a bounded sample of
the same workload (N = 1 only; cpu_baseline is null on a multi-GPU line).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference] [--no-extras]
Multi-GPU: torchrun --nproc-per-node N bench.py --gpus N  (sample sharding: every rank evaluates
the same population on its own 2^20 samples and one int32 all-reduce per step sums the counts:
weak scaling).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "condition-evals/s & rule-set·samples/s vs plain; p50/p99 served latency"
UNIT = "condition-evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "hard_eval_counters.json")


# ----------------------------------------------------------------------------- helpers

def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# evaluator kernel of each tile-configuration version (finite, ranked datasets)
KERNEL_OF_VERSION = {1: "k_hard", 2: "k_hard2", 3: "k_hard2", 4: "k_hard4", 5: "k_hard5"}


def hard_algorithmic_ops(batch, N):
    """Algorithmic lane operations of one evaluation: 1 compare per threshold condition-eval,
    2 multiplies + 1 compare per pair condition-eval, and per rule 3 word operations (AND,
    AND-NOT, popcount) per 32 samples."""
    n_pair = int((batch.cond_g >= 0).sum())
    n_thr = batch.C - n_pair
    return N * (n_thr + 3 * n_pair) + 3 * batch.R * ((N + 31) // 32)


def executed_work(prof, batch, N):
    """The rank-coded evaluator's own count of the work it did (one call in a work-counting
    context, RS_CTX_COUNT_WORK): per launch, the records walked (one per condition, 128 samples each), the pair / product /
    membership rows among them and the rule ends, as algorithmic operations counted like
    hard_algorithmic_ops (1 per threshold sample, 3 per pair sample, 3 word operations per rule
    end per 32 samples), and the share of the nominal records that were walked."""
    n = max(1, prof.get("counted_launches", 0))
    rec = prof.get("hard_records_walked", 0) / n
    if rec <= 0:
        return None
    rows = prof.get("hard_rows_walked", 0) / n
    ends = prof.get("hard_rule_ends_walked", 0) / n
    tiles = (N + 127) // 128
    return {"ops_per_launch": 128 * ((rec - rows) + 3 * rows) + 12 * ends,
            "records_walked_per_launch": rec,
            "records_walked_share": rec / (batch.C * tiles),
            "set_tiles_per_launch": prof.get("hard_set_tiles", 0) / n}


def source_hash():
    h = hashlib.sha256()
    for f in ("hard_eval.cu", "hard_eval4.cu", "hard_eval5.cu", "eval_rank.cuh", "eval_core.cuh", "pack.cu",
              "rs_internal.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_2406_01821_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_counters():
    """The committed ncu summary of the evaluator if it was taken on the current kernel source
    (else None): DRAM bytes per launch and the utilisation of its bottleneck pipes."""
    try:
        with open(PROFILE_SUMMARY) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d


# ----------------------------------------------------------------------------- CPU oracle

def cpu_baseline(w, n_sample: int, threads: int = 0, single_thread: bool = False):
    import oracle
    Xs, ys = w.X[:n_sample], w.y[:n_sample]
    nt = oracle.num_threads(threads)
    oracle.eval_hard(Xs[:256], ys[:256], w.K, w.batch, nthreads=nt)      # warm
    t0 = time.perf_counter()
    oracle.eval_hard(Xs, ys, w.K, w.batch, nthreads=nt)
    dt = time.perf_counter() - t0
    v = w.batch.nominal_conditions() * n_sample / dt
    out = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle",
           "sample": f"all {w.batch.P} sets on the first {n_sample} of {w.N} samples "
                     f"({dt:.2f} s wall, OpenMP over sets)"}
    if single_thread and nt > 1:        # the same oracle on one core, on a sample a sixteenth the size
        n1 = max(256, n_sample // 16)
        t0 = time.perf_counter()
        oracle.eval_hard(Xs[:n1], ys[:n1], w.K, w.batch, nthreads=1)
        d1 = time.perf_counter() - t0
        out["single_thread"] = {"value": w.batch.nominal_conditions() * n1 / d1, "cores": 1,
                                "sample": f"all {w.batch.P} sets on the first {n1} samples ({d1:.2f} s wall)"}
    return out


# ----------------------------------------------------------------------------- legs

def hard_leg(args, rank, dev, ctx_mod, w):
    import torch
    from paper_2406_01821_gb300 import rs
    stream = torch.cuda.Stream(device=dev)
    ctx = rs.Context(dev, flags=rs.CTX_PROFILE)
    ds = ctx.dataset(w.X, w.y, w.K)
    db = rs.DeviceBatch.from_host(w.batch, device=f"cuda:{dev}")
    if args.tile is not None:
        tile = args.tile
    else:
        tile = 0 if args.no_autotune else ctx.autotune(ds, db, stream=stream)
    if args.no_autotune or args.tile is not None:
        ctx.set_tile_config(tile)
    P, K, N = w.batch.P, w.K, w.N
    counts = torch.empty(P + P * K, dtype=torch.int32, device=dev)
    out = (counts[:P], counts[P:].view(P, K), None)

    def step():
        ctx.eval_hard(ds, db, K, out=out, stream=stream)
        if ctx_mod.world > 1:          # sample sharding: the one exchange step, on the same stream
            with torch.cuda.stream(stream):
                ctx_mod.pg.all_reduce(counts)
    for _ in range(args.warmup):
        step()
    stream.synchronize()
    ctx_mod.barrier()
    ctx.profile(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        e1.synchronize()
    ctx_mod.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile(reset=True)
    correct = out[0].cpu().numpy()

    # end to end through the public call with pinned host buffers (copies inside the region)
    hb = rs.HostBatch(w.batch)
    pinned = {}
    for f, a in hb.a.items():
        if a is None:
            continue
        t = torch.empty(a.shape, dtype=torch.from_numpy(a).dtype, pin_memory=True)
        t.numpy()[...] = a
        pinned[f] = t
    hb.a = {f: (pinned[f].numpy() if f in pinned else None) for f in hb.a}
    hc = torch.empty(P, dtype=torch.int32, pin_memory=True).numpy()
    hpc = torch.empty((P, K), dtype=torch.int32, pin_memory=True).numpy()
    ctx2 = rs.Context(dev)
    ds2 = ctx2.dataset(w.X, w.y, w.K)
    from paper_2406_01821_gb300.rs import check, lib, _ptr, _stream_ptr
    import ctypes
    cb = hb.c()

    # several GPUs: the sharded evaluation's exchange step on the host results (up, one int32
    # all-reduce, down), as the sample-sharded call does it
    red = torch.empty(P + P * K, dtype=torch.int32, device=dev) if ctx_mod.world > 1 else None

    def e2e_call():
        check(lib().rs_eval_hard(ctx2.h, ds2, ctypes.byref(cb), _ptr(hc), _ptr(hpc), None,
                                 _stream_ptr(stream)))
        if red is not None:
            with torch.cuda.stream(stream):
                red[:P].copy_(torch.from_numpy(hc))
                red[P:].copy_(torch.from_numpy(hpc).view(-1))
                ctx_mod.pg.all_reduce(red)
                hc[...] = red[:P].cpu().numpy()
                hpc[...] = red[P:].view(P, K).cpu().numpy()
    for _ in range(max(1, args.warmup)):
        e2e_call()
    stream.synchronize()
    ctx_mod.barrier()
    t0 = time.perf_counter()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        e2e_call()
    f1.record(stream)
    f1.synchronize()
    e2e_ms = max(f0.elapsed_time(f1), (time.perf_counter() - t0) * 1e3) / args.steps
    e2e_ok = bool(np.array_equal(hc, correct))       # several GPUs: both are the summed counts
    ctx2.close()
    # one more call, untimed, in a context whose evaluator counts the work it does
    ctx3 = rs.Context(dev, flags=rs.CTX_COUNT_WORK | rs.CTX_NO_GRAPH)
    ds3 = ctx3.dataset(w.X, w.y, w.K)
    ctx3.set_tile_config(tile)
    ctx3.profile(reset=True)
    ctx3.eval_hard(ds3, db, K, out=out, stream=stream)
    stream.synchronize()
    walked = ctx3.profile(reset=True)
    ctx3.close()
    for f in ("hard_records_walked", "hard_rows_walked", "hard_rule_ends_walked", "hard_set_tiles"):
        prof[f] = walked[f]
    prof["counted_launches"] = 1
    ctx.close()
    xfer = 0 if red is None else red.numel() * 4      # the exchange's own copies
    return {"ms": ms, "prof": prof, "tile": tile, "clocks": clk.summary(), "e2e_ms": e2e_ms,
            "e2e_ok": e2e_ok, "h2d": hb_nbytes(hb) + xfer, "d2h": hc.nbytes + hpc.nbytes + xfer}


def hb_nbytes(hb):
    return int(sum(a.nbytes for a in hb.a.values() if a is not None))


def soft_leg(args, dev):
    import torch
    from paper_2406_01821_gb300 import rs, synth
    if args.workload == "soft-small":
        w = synth.soft_tune(seed=0, N=65536, P=256)
    else:
        w = synth.soft_tune(seed=0)
    ctx = rs.Context(dev, flags=rs.CTX_PROFILE)
    stream = torch.cuda.Stream(device=dev)
    ds = ctx.dataset(w.X, w.y, w.K)
    db = rs.DeviceBatch.from_host(w.batch, device=f"cuda:{dev}")
    dl = torch.ones(w.batch.P, device=dev)
    steps = max(1, args.steps // 5)
    for _ in range(1):
        ctx.soft_bwd(ds, db, w.tau, dl, stream=stream)
    stream.synchronize()
    ctx.profile(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.soft_bwd(ds, db, w.tau, dl, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = ctx.profile(reset=True)
    rates = ctx.pipe_rates()
    ctx.close()
    cs = w.batch.nominal_conditions() * w.N
    kern_ms = prof["soft_ms"] / max(1, prof["soft_launches"])
    xu = soft_transcendentals(w.batch, w.N)
    xu_peak = rates["ex2"]
    return {"workload": w.name, "ms_per_step": ms, "condition_samples_per_s": cs / (ms / 1e3),
            "rule_set_samples_per_s": w.batch.P * w.N / (ms / 1e3),
            "kernel_ms": kern_ms, "steps": steps,
            "what": "forward + adjoint (loss and gradients w.r.t. a, b, t of every condition)",
            "roofline": {"bound": "xu", "achieved": xu / (kern_ms / 1e3) / 1e12, "peak": xu_peak / 1e12,
                         "unit": "T transcendentals/s", "frac": xu / (kern_ms / 1e3) / xu_peak,
                         "transcendentals_per_pass": xu,
                         "peak_source": "measured: special-function unit ex2 stream (rs_measure_pipe_rates)"}}


def categorical_leg(args, dev):
    """The ragged workload's shape with a quarter of the features categorical (48 codes): every
    condition on those features is a membership test. Hard evaluation, device-resident inputs."""
    import torch
    import oracle
    from paper_2406_01821_gb300 import rs, synth
    N = (1 << 19) if args.workload == "ragged-small" else (1 << 20)
    P = 512 if args.workload == "ragged-small" else 4096
    F, K, n_cat = 128, 10, 32
    X, y = synth.categorical_mixture(N, F, K, 0, n_cat=n_cat, n_codes=48)
    b = synth.random_rulesets(synth.quantile_table(X), K, P, (1, 64), (1, 8), 0, cat_from=F - n_cat, n_codes=48)
    ctx = rs.Context(dev, flags=rs.CTX_PROFILE)
    stream = torch.cuda.Stream(device=dev)
    ds = ctx.dataset(X, y, K)
    db = rs.DeviceBatch.from_host(b, device=f"cuda:{dev}")
    out = (torch.empty(P, dtype=torch.int32, device=dev), torch.empty((P, K), dtype=torch.int32, device=dev), None)
    for _ in range(max(1, args.warmup)):
        ctx.eval_hard(ds, db, K, out=out, stream=stream)
    stream.synchronize()
    ctx.profile(reset=True)
    steps = max(1, args.steps // 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.eval_hard(ds, db, K, out=out, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = ctx.profile(reset=True)
    ctx.close()
    nominal = b.nominal_conditions() * N
    n_s = 1024
    nt = oracle.num_threads(0)
    t0 = time.perf_counter()
    oracle.eval_hard(X[:n_s], y[:n_s], K, b, nthreads=nt)
    dt = time.perf_counter() - t0
    return {"workload": f"categorical P={P} R=1..64 C=1..8 N={N} F={F} ({n_cat} categorical, 48 codes) K={K}",
            "metric": METRIC, "value": nominal / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "membership_conditions": int((b.cond_op == synth.IN).sum()), "conditions": int(b.C),
            "kernel_ms": prof["hard_ms"] / max(1, prof["hard_launches"]),
            "cpu_baseline": {"value": b.nominal_conditions() * n_s / dt, "unit": UNIT, "cores": nt,
                             "kind": "oracle", "sample": f"all {P} sets on the first {n_s} samples ({dt:.2f} s)"}}


def plain_leg(args, dev):
    """The paper's experiment shape (569 samples x 30 features, 64 sets x 8 rules x 1..3
    conditions), with the outputs that shape names: per-sample predictions [P][N] and per-set
    correct counts (and, beside it, the counts alone). Launch-bound, so reported as time per call
    and evaluations per second, with no roofline fraction."""
    import torch
    from paper_2406_01821_gb300 import rs, synth
    w = synth.plain_hard(seed=0)
    ctx = rs.Context(dev)
    stream = torch.cuda.Stream(device=dev)
    ds = ctx.dataset(w.X, w.y, w.K)
    db = rs.DeviceBatch.from_host(w.batch, device=f"cuda:{dev}")
    P, K = w.batch.P, w.K
    reps = 200

    def per_call(out):
        for _ in range(20):
            ctx.eval_hard(ds, db, K, out=out, stream=stream)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.eval_hard(ds, db, K, out=out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    correct = torch.empty(P, dtype=torch.int32, device=dev)
    pc = torch.empty((P, K), dtype=torch.int32, device=dev)
    preds = torch.empty((P, w.N), dtype=torch.int32, device=dev)
    us = per_call((correct, pc, preds))
    us_counts = per_call((correct, pc, None))
    ctx.close()
    return {"workload": w.name, "outputs": "predictions [P][N], correct [P], per-class counts [P][K]",
            "us_per_call": us, "condition_evals_per_s": w.nominal_cond_evals() / (us * 1e-6),
            "rule_set_samples_per_s": P * w.N / (us * 1e-6), "calls": reps,
            "us_per_call_counts_only": us_counts,
            "note": "launch-bound (pack + validate + evaluate: one cached graph replayed per call); no roofline fraction"}


def soft_transcendentals(batch, N):
    """Algorithmic transcendentals of one forward + adjoint pass, as the method states them: per
    condition and sample an exp and a log1p (log-sigmoid) and an exp (sigmoid of -u); per rule and
    sample an expm1 and a log (log(1 - q)) forward and again in the adjoint, an exp (the gradient
    of lq), two log-sum-exps (exp + log1p each) in the adjoint and one forward for rules of the
    sample's class (counted for every rule: an upper bound on the forward share). The kernels do
    fewer per rule: the adjoint reuses the forward's log(1 - q) and runs one of its two
    log-sum-exps (the other only adds log(1 - q))."""
    return N * (3 * batch.C + 11 * batch.R)


def evolution_leg(args, dev, G: int = 200, arms: bool = True):
    """Device-resident evolution: population 10,000 (R <= 32, C <= 6), 200 generations on
    N=100,000 x F=32 two-class data, the best 64 fine-tuned (50 Adam steps) every 10 generations.
    Compared with two plain arms per generation: the CPU oracle (evaluation + evolution on the host
    cores) and host-driven evolution with one GPU evaluation launch per generation (arms=False:
    the device loop alone, e.g. G=10 for a launch list of one fine-tuning round)."""
    import torch
    from paper_2406_01821_gb300 import rs, synth
    X, y = synth.evolution_data(seed=0)
    P, RMAX, CMAX = 10000, 32, 6
    pop = synth.initial_population(X, y, 2, P, RMAX, CMAX, seed=0)
    ctx = rs.Context(dev)
    ds = ctx.dataset(X, y, 2)
    stream = torch.cuda.Stream(device=dev)
    ctx.evolve(ds, pop, generations=2, elite=100, seed=1, stream=stream)          # warm-up
    t0 = time.perf_counter()
    _, fit, best, mean = ctx.evolve(ds, pop, generations=G, elite=100, seed=1, tune_every=10,
                                    tune_top=64, tune_steps=50, tau=0.1, lr=1e-2, stream=stream)
    t_tuned = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.evolve(ds, pop, generations=G, elite=100, seed=1, stream=stream)
    t_plain_gpu = time.perf_counter() - t0
    if not arms:
        ctx.close()
        return {"workload": f"evolution P={P} R<=32 C<=6 N={len(X)} F=32 K=2 generations={G} "
                            "tune top-64 x 50 Adam steps every 10",
                "generations_per_s": G / t_tuned, "generations_per_s_without_tuning": G / t_plain_gpu}
    import oracle                 # the plain arms: the oracle's evolution step on the host
    # host-driven arm: one evaluation launch per generation, evolution on the host
    hb_gens = 3
    t0 = time.perf_counter()
    cur = pop
    for g in range(hb_gens):
        b = synth.batch_from_population(cur)
        c, _, _ = ctx.eval_hard(ds, rs.HostBatch(b), 2, per_class=False)
        cur = oracle.evolve_step(cur, c, 1, g, 100, X, 2)
    t_host = (time.perf_counter() - t0) / hb_gens
    # CPU arm: the oracle evaluates and evolves (one generation, all host cores)
    t0 = time.perf_counter()
    c, _, _ = oracle.eval_hard(X, y, 2, synth.batch_from_population(pop), want_per_class=False)
    oracle.evolve_step(pop, c, 1, 0, 100, X, 2)
    t_cpu = time.perf_counter() - t0
    ctx.close()
    return {"workload": f"evolution P={P} R<=32 C<=6 N={len(X)} F=32 K=2 generations={G} "
                        "tune top-64 x 50 Adam steps every 10",
            "generations_per_s": G / t_tuned, "seconds": t_tuned,
            "generations_per_s_without_tuning": G / t_plain_gpu,
            "best_first_last": [int(best[0]), int(best[-1])], "mean_last": float(mean[-1]),
            "plain_host_driven_gpu_generations_per_s": 1.0 / t_host,
            "plain_cpu_oracle_generations_per_s": 1.0 / t_cpu,
            "cpu_cores": oracle.num_threads(0)}


SERVE_LOADS = (0.7, 1.0, 1.3)


def serving_leg(args, dev):
    """Continuous batching of fitness requests from 256 concurrent evolution runs (each with its own
    resident dataset: N log-uniform [500, 500000], F ~ U{8..256}, K ~ U{2..10}); request
    populations P log-uniform [16, 2048], R ~ U{1..64}, C ~ U{1..8}; 40 GB budget. Poisson
    arrivals at 0.7, 1.0 and 1.3 of the measured capacity of the plain one-request-per-launch
    evaluator. Latency = completion - arrival, for the served path and for the plain evaluator
    (FIFO, one launch per request) on the same GPU and the same arrival times."""
    import queue
    import torch
    from paper_2406_01821_gb300 import rs, synth
    runs_N, runs_F, runs_K = synth.serving_runs(seed=0, runs=256)
    ctx = rs.Context(dev, mem_budget_bytes=40 << 30)
    dss, qtabs = [], []
    for i in range(len(runs_N)):
        X, y = synth.gaussian_mixture(int(runs_N[i]), int(runs_F[i]), int(runs_K[i]), 1000 + i)
        dss.append(ctx.dataset(X, y, int(runs_K[i])))
        qtabs.append(synth.quantile_table(X, m=4096))
        del X, y
    M = args.serve_requests
    rng = np.random.default_rng(7)
    Ps = synth.serving_request_sizes(seed=0, count=M)
    reqs = []
    for j in range(M):
        i = int(rng.integers(0, len(runs_N)))
        b = synth.random_rulesets(qtabs[i], int(runs_K[i]), int(Ps[j]), (1, 64), (1, 8), 5000 + j)
        reqs.append((i, rs.HostBatch(b), b.nominal_conditions() * int(runs_N[i])))
    total = float(sum(r[2] for r in reqs))
    # plain capacity: the mean service time of the whole request mix evaluated back to back, one
    # launch per request (request sizes are heavy-tailed: a subset's mean is a biased estimate)
    for j in range(8):
        i, hb, _ = reqs[j]
        ctx.eval_hard(dss[i], hb, int(runs_K[i]))
    t0 = time.perf_counter()
    for (i, hb, _) in reqs:
        ctx.eval_hard(dss[i], hb, int(runs_K[i]))
    service = (time.perf_counter() - t0) / M
    for j in range(8):            # warm-up of the served path: scheduler, kernel, staging pool
        i, hb, _ = reqs[j]
        ctx.poll(ctx.submit(dss[i], hb), hb.P, int(runs_K[i]), timeout_us=60_000_000)

    def drive(arrivals, submit, finish_all):
        t_start = time.perf_counter() + 0.05
        for j in range(M):
            wait = t_start + arrivals[j] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            submit(j, t_start + arrivals[j])
        return finish_all(), t_start

    def summ(lat, dur):
        a = np.array(lat) * 1e3
        return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                "mean_ms": float(a.mean()), "requests_per_s": M / dur, "condition_evals_per_s": total / dur}

    def at_load(load, seed):
        arrivals = np.cumsum(np.random.default_rng(seed).exponential(service / load, size=M))
        # plain: FIFO worker, one rs_eval_hard launch per request
        q = queue.Queue()
        lat_plain = [0.0] * M

        def worker():
            while True:
                item = q.get()
                if item is None:
                    return
                j, t_arr = item
                i, hb, _ = reqs[j]
                ctx.eval_hard(dss[i], hb, int(runs_K[i]))
                lat_plain[j] = time.perf_counter() - t_arr
        th = threading.Thread(target=worker)
        th.start()

        def fin_plain():
            q.put(None)
            th.join()
            return time.perf_counter()
        t_end, t_start = drive(arrivals, lambda j, ta: q.put((j, ta)), fin_plain)
        dur_plain = t_end - t_start
        # served: rs_submit at arrival, completion times from the library's ticket info
        tickets = [0] * M
        t_arr_ns = [0] * M

        def submit(j, ta):
            i, hb, _ = reqs[j]
            tickets[j] = ctx.submit(dss[i], hb)
            t_arr_ns[j] = time.monotonic_ns() - int((time.perf_counter() - ta) * 1e9)

        lat_srv = [0.0] * M
        split = np.zeros((M, 3))      # arrival -> submit returned, -> admitted, -> done (seconds)

        def fin_served():
            for j in range(M):
                i, hb, _ = reqs[j]
                out = ctx.poll(tickets[j], hb.P, int(runs_K[i]), timeout_us=120_000_000)
                lat_srv[j] = (out[2]["done_ns"] - t_arr_ns[j]) / 1e9
                split[j] = [(out[2]["submit_ns"] - t_arr_ns[j]) / 1e9,
                            (out[2]["admit_ns"] - out[2]["submit_ns"]) / 1e9,
                            (out[2]["done_ns"] - out[2]["admit_ns"]) / 1e9]
            return time.perf_counter()
        t_end, t_start = drive(arrivals, submit, fin_served)
        dur_srv = t_end - t_start
        pct = lambda c, q_: float(np.percentile(split[:, c], q_) * 1e3)
        return {"offered_load_x_plain_capacity": load, "arrival_rate_per_s": load / service,
                "served": summ(lat_srv, dur_srv), "plain_one_launch_per_request": summ(lat_plain, dur_plain),
                "served_p50_split_ms": {"arrival_to_queued": pct(0, 50), "queued_to_admitted": pct(1, 50),
                                        "admitted_to_done": pct(2, 50)},
                "served_p99_split_ms": {"arrival_to_queued": pct(0, 99), "queued_to_admitted": pct(1, 99),
                                        "admitted_to_done": pct(2, 99)}}

    sweep = [at_load(load, 7 + k) for k, load in enumerate(SERVE_LOADS)]
    # capacity: every request at once (served) / back to back (plain)
    t0 = time.perf_counter()
    ts = [ctx.submit(dss[i], hb) for (i, hb, _) in reqs]
    for j, t in enumerate(ts):
        i, hb, _ = reqs[j]
        ctx.poll(t, hb.P, int(runs_K[i]), timeout_us=300_000_000)
    burst_srv = time.perf_counter() - t0
    t0 = time.perf_counter()
    for (i, hb, _) in reqs:
        ctx.eval_hard(dss[i], hb, int(runs_K[i]))
    burst_plain = time.perf_counter() - t0
    stats = ctx.serving_stats()
    ctx.close()
    return {"workload": f"serving {M} requests from 256 runs, Poisson arrivals at "
                        f"{', '.join(str(x) for x in SERVE_LOADS)} x plain capacity, 40 GB budget",
            "plain_service_ms": service * 1e3, "sweep": sweep,
            "persistent_kernel_launches": stats["kernel_launches"],
            "capacity_condition_evals_per_s": {"served_all_at_once": total / burst_srv,
                                               "plain_back_to_back": total / burst_plain}}


# ----------------------------------------------------------------------------- distributed

class Dist:
    """Ranks of a torchrun launch (one per GPU, NCCL); a single process otherwise. Without CUDA
    (multi-rank tests on the CPU) the ranks use gloo and CPU tensors."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.dev = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local)
                self.dev = f"cuda:{self.local}"
                dist.init_process_group("nccl", device_id=torch.device(self.dev))
            else:
                dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def _reduce(self, v: float, op) -> float:
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.dev)
        self.pg.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v: float) -> float:
        return self._reduce(v, self.pg.ReduceOp.MAX) if self.pg else v

    def sum(self, v: float) -> float:
        return self._reduce(v, self.pg.ReduceOp.SUM) if self.pg else v

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def whole_job_rate(d: Dist, units: float, ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling: every rank
    evaluates the population on its own samples)."""
    return d.sum(units) / (d.max(ms) / 1e3)


# ----------------------------------------------------------------------------- main

def run_reference(args, d: Dist):
    """The reference arm: the CPU oracle as it stands, on bounded samples of the workload."""
    if d.rank != 0:
        return
    from paper_2406_01821_gb300 import synth
    w = synth.ragged_hard(seed=0)
    n_sample = min(args.cpu_sample, 131072)      # about 2.5 s of oracle work per step on 16 cores
    for _ in range(args.warmup):
        cpu_baseline(w, min(n_sample, 4096))
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, n_sample))
    dt = (time.perf_counter() - t_all) / args.steps
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": w.name, "sample_per_step": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def parse_skip(text: str) -> set:
    """Names of the extra legs to skip, from a comma-separated list (whole names only)."""
    return {x.strip() for x in (text or "").split(",") if x.strip()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=524288)
    ap.add_argument("--workload", default="ragged", choices=["ragged", "ragged-small", "soft-small", "evolution-small"],
                    help="ragged-small (N=2^19, P=512), soft-small (soft leg only, N=65536, P=256) and "
                         "evolution-small (the evolution loop alone, 10 generations: one fine-tuning "
                         "round) are the cases used for ncu captures")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile", type=int, default=None, help="force a tile configuration id")
    ap.add_argument("--skip", default="", help="comma-separated extra legs to skip (soft,evolution,serving,categorical,plain)")
    ap.add_argument("--serve-requests", type=int, default=512)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    d = Dist()
    if args.impl == "reference":
        run_reference(args, d)
        d.close()
        return

    import torch
    from paper_2406_01821_gb300 import build, rs, synth
    if d.rank == 0 or d.world == 1:
        build.build()
    d.barrier()
    dev = d.local
    torch.cuda.set_device(dev)
    if args.workload == "soft-small":
        print(json.dumps({"soft": soft_leg(args, dev)}), flush=True)
        d.close()
        return
    if args.workload == "evolution-small":
        print(json.dumps({"evolution": evolution_leg(args, dev, G=10, arms=False)}), flush=True)
        d.close()
        return
    if args.workload == "ragged-small":
        w = synth.ragged_hard(seed=0, N=1 << 19, P=512)
    else:
        w = synth.ragged_hard(seed=0)
    if d.world > 1 and d.rank > 0:
        # sample sharding: every rank evaluates the same population on its own samples (rank r's
        # rows drawn from the mixture generator with seed r); the counts are summed by one
        # all-reduce per step
        X, y = synth.gaussian_mixture(w.N, w.F, w.K, d.rank)
        w = dataclasses.replace(w, X=X, y=y)
    res = hard_leg(args, d.rank, dev, d, w)
    ms_max = d.max(res["ms"])
    e2e_max = d.max(res["e2e_ms"])
    nominal = w.batch.nominal_conditions() * w.N
    total_nominal = d.sum(float(nominal))
    total_sets = float(w.batch.P)
    value = whole_job_rate(d, float(nominal), res["ms"])

    prof = res["prof"]
    kern_ms = prof["hard_ms"] / max(1, prof["hard_launches"])
    ops = hard_algorithmic_ops(w.batch, w.N)
    executed = executed_work(prof, w.batch, w.N)
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ops = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    with rs.Context(dev) as pctx:
        rates = pctx.pipe_rates()
    counters = profiled_counters()
    traffic = counters.get("dram_bytes_per_launch_full") if counters else None
    pipes = ({"issue_active": counters["issue_active_pct"] / 100, "l1tex_throughput": counters["l1tex_throughput_pct"] / 100,
              "alu_pipe": counters["alu_pipe_pct"] / 100, "source": "profiles/hard_eval_k_hard5_full.md (N=2^19)"}
             if counters and "issue_active_pct" in counters else None)
    extras = {}
    # the extra legs and the CPU baseline run at N = 1 only (a multi-GPU launch holds every GPU
    # while rank 0 would run them)
    if not args.no_extras and d.world == 1:
        skip = parse_skip(args.skip)
        for name, leg in (("soft", soft_leg), ("evolution", evolution_leg),
                          ("serving", serving_leg), ("categorical", categorical_leg), ("plain", plain_leg)):
            if name in skip:
                continue
            try:
                extras[name] = leg(args, dev)
            except Exception as e:     # an extra leg never hides the headline number
                extras[name] = {"error": repr(e)}

    if d.rank == 0:
        cb = cpu_baseline(w, args.cpu_sample, single_thread=True) if d.world == 1 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "global_batch": int(total_sets), "samples": w.N * d.world,
                       "features": w.F, "classes": w.K,
                       "nominal_cond_evals_per_step": int(total_nominal),
                       "tile_config": rs.tile_configs()[res["tile"]],
                       "l2": "inputs larger than L2 (feature-major dataset 512 MiB per GPU)",
                       "parallelism": ("one GPU" if d.world == 1 else
                                       f"samples per GPU x{d.world}, one int32 all-reduce of the counts per step")},
            "rule_set_samples_per_s": total_sets * w.N * d.world / (ms_max / 1e3),
            "roofline": {"bound": "alu", "achieved": ops / (kern_ms / 1e3) / 1e12,
                         "peak": peak_ops / 1e12, "unit": "Tops/s",
                         "frac": (ops / (kern_ms / 1e3)) / peak_ops, "traffic": traffic,
                         "kernel": KERNEL_OF_VERSION.get(rs.tile_configs()[res["tile"]]["form"], "k_hard"),
                         "kernel_ms": kern_ms,
                         "ops_per_launch": ops, "bottleneck_pipes": pipes,
                         "executed": None if executed is None else {
                             **executed, "frac": executed["ops_per_launch"] / (kern_ms / 1e3) / peak_ops},
                         "peak_source": f"{sms} SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                        f"({peak_src} max clock)",
                         "measured_pipes_T_lane_ops": {k: v / 1e12 for k, v in rates.items()}},
            "cpu_baseline": cb,
            "e2e": {"value": total_nominal / (e2e_max / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"],
                    "ms_per_step": e2e_max, "matches_device_run": res["e2e_ok"]},
            "clocks": res["clocks"],
            "gpu_launches": int(prof["launches"]),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    d.close()


if __name__ == "__main__":
    main()
