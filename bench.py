#!/usr/bin/env python
"""Throughput of GB300 spectral-bound coarsening (M fine edges/s per coarsening level).

One step = one full coarsening of the workload (every level: validation, degrees, normalised
rows, scores, merge selection, relabel, contraction), inputs resident in HBM.  The default
workload (the headline) is the largest single graph: a random geometric graph of 2^23 points
in the unit cube, mean degree 12, FP32 weights exp(-d^2/r^2), coarsened by eight halving
levels to n/256.  value = (sum over levels of the fine edges that level processed) / (device
time of a step).  The same line carries, under "configs", the other configurations: the
2048x2048 FP64 triangle mesh (6 levels), the 129^3 FP64 tetrahedral mesh (7 levels), the
random geometric graph coarsened in one level to n/256, and the 10,000-mesh batch (forward +
backward graphs/s against a per-graph loop).  Under torchrun each rank coarsens its own
replica (the single-graph path does not shard), so value is the sum over ranks; the batch
shards by graphs.

--impl reference times the CPU oracle instead (test infrastructure, the only other use of it
here), on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "M fine edges/s per coarsening level"
UNIT = "M edges/s"

WORKLOADS = {
    # name: (config name, levels, description)
    "c2_tri2048_f64": ("c2_tri2048_f64", 6, "2048x2048 jittered triangle mesh (4,194,304 nodes, "
                       "12,574,721 edges), FP64 weights 1/edge-length, 6 halving levels to n/64"),
    "c3_tet129_f64": ("c3_tet129_f64", 7, "129^3-vertex tetrahedral cube mesh (2,146,689 nodes, "
                      "14,827,904 edges), FP64 1/edge-length, 7 halving levels to n/128"),
    "c4_rgg8m_f32": ("c4_rgg8m_f32", 8, "random geometric graph, 2^23 points, mean degree 12, "
                     "FP32 exp(-d^2/r^2), 8 halving levels to n/256"),
    "c4_rgg8m_f32_one": ("c4_rgg8m_f32_one", 1, "random geometric graph, 2^23 points, mean "
                         "degree 12, FP32 exp(-d^2/r^2), one level to n/256"),
    "c4_rgg8m_f32_reordered": ("c4_rgg8m_f32", 8, "random geometric graph, 2^23 points, mean "
                               "degree 12, FP32 exp(-d^2/r^2), 8 halving levels to n/256, "
                               "with the adjacency-reordering option: renumbered by "
                               "(8-hop min label, 2-hop min label, id) inside the timed step"),
    # reduced case of the same construction, for profiler captures that must stay small
    "p2_tri512_f64": ("p2_tri512_f64", 6, "512x512 jittered triangle mesh (262,144 nodes, "
                      "784,385 edges), FP64 1/edge-length, 6 halving levels to n/64"),
    "p4_rgg2m_f32": ("p4_rgg2m_f32", 8, "random geometric graph, 2^21 points, mean degree 12, "
                     "FP32 exp(-d^2/r^2), 8 halving levels to n/256"),
}
# the CPU oracle's bounded sample: the same construction at a quarter of the side length
SAMPLES = {
    "c2_tri2048_f64": dict(kind="tri", nx=512, ny=512, jitter=0.3, weight="inv_len",
                           dtype="float64", seed=2, ratio=64),
    "c3_tet129_f64": dict(kind="tet", k=33, jitter=0.25, weight="inv_len", dtype="float64",
                          seed=3, ratio=128),
    "c4_rgg8m_f32": dict(kind="rgg", n=1 << 17, degree=12.0, dtype="float32", seed=4, ratio=256),
    "c4_rgg8m_f32_one": dict(kind="rgg", n=1 << 17, degree=12.0, dtype="float32", seed=4,
                             ratio=256, mode="one"),
    "c4_rgg8m_f32_reordered": dict(kind="rgg", n=1 << 17, degree=12.0, dtype="float32", seed=4,
                                   ratio=256, reorder=True),
    "p2_tri512_f64": dict(kind="tri", nx=256, ny=256, jitter=0.3, weight="inv_len",
                          dtype="float64", seed=12, ratio=64),
    "p4_rgg2m_f32": dict(kind="rgg", n=1 << 16, degree=12.0, dtype="float32", seed=4, ratio=256),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _sample_graph(spec):
    from paper_2204_11757_gb300 import inputs as I
    dt = np.dtype(spec["dtype"])
    if spec["kind"] == "tri":
        return I.tri_mesh_2d(spec["nx"], spec["ny"], spec["seed"], spec["jitter"], spec["weight"],
                             dt)
    if spec["kind"] == "tet":
        return I.tet_mesh_3d(spec["k"], spec["seed"], spec["jitter"], spec["weight"], dt)
    return I.rgg_3d(spec["n"], spec["degree"], spec["seed"], dt)


def _oracle_step(g, spec):
    """One oracle coarsening of the sample; returns (fine edges processed, seconds)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    if spec.get("reorder"):
        levels, _, _ = O.coarsen_reordered(g, spec["ratio"], spec.get("mode", "halving"))
    else:
        levels, _ = O.coarsen(g, spec["ratio"], spec.get("mode", "halving"))
    dt = time.perf_counter() - t0
    return sum(lv.f.shape[0] for lv in levels), dt


def _score_rate(g, fn, budget_s):
    """M edges/s of one score function (S1-S3) repeated for about budget_s on the sample."""
    done, t, runs = 0, 0.0, 0
    while t < budget_s or runs == 0:
        t0 = time.perf_counter()
        out = fn(g)
        t += time.perf_counter() - t0
        done += g.m
        runs += 1
    return done / t / 1e6, out


def _host():
    """The host the CPU numbers were taken on: its hardware threads and processor model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model}


def cpu_baseline(workload, budget_s=10.0):
    from oracle import oracle as O
    spec = SAMPLES[workload]
    g = _sample_graph(spec)
    edges, dt, runs = 0, 0.0, 0
    while dt < budget_s or runs == 0:
        e, t = _oracle_step(g, spec)
        edges += e
        dt += t
        runs += 1
    # the score step alone: sequential, and with the edges split over every host thread (the
    # parallel fitness loop of Algorithm 1 on a CPU; same bits)
    seq, _ = _score_rate(g, O.score, 2.0)
    par, (_, threads) = _score_rate(g, O.score_parallel, 2.0)
    return {"value": edges / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"full {spec.get('mode', 'halving')} coarsening (ratio {spec['ratio']}) of "
                      f"the same construction at reduced size: n={g.n}, m={g.m}; {runs} runs, "
                      f"{dt:.1f} s single-threaded C",
            "score_step": {"unit": "M edges/s", "sequential": seq, "parallel": par,
                           "parallel_threads": threads,
                           "sample": f"level-0 scores (S1-S3) of the same sample, ~2 s each"},
            "host": _host()}


def _oracle_batch_sample():
    """A 60-graph sample of the 10,000-mesh batch and a timer of the oracle on it (each graph
    coarsened in 3 levels, then its contraction gradient)."""
    from oracle import oracle as O
    from paper_2204_11757_gb300 import inputs as I
    full, cfg = I.config_graph("c5_batch10k_f32")
    rng = np.random.default_rng(0)
    sub = I.subsample_batch(full, np.sort(rng.choice(full.B, size=60, replace=False)))

    def one():
        t0 = time.perf_counter()
        for levels, _ in O.coarsen_batch(sub, cfg["ratio"], cfg["mode"]):
            em = O.compose_emaps(levels)
            O.contract_backward(em, np.ones(levels[-1].coarse.m_c, dtype=np.float32))
        return time.perf_counter() - t0
    return sub, one


def _oracle_batched(budget_s=10.0):
    sub, one = _oracle_batch_sample()
    t, runs = 0.0, 0
    while t < budget_s or runs == 0:
        t += one()
        runs += 1
    return {"value": sub.B * runs / t, "unit": "graphs/s", "cores": 1, "kind": "oracle",
            "sample": f"{sub.B} sampled graphs of the batch, {runs} runs, {t:.1f} s "
                      f"single-threaded C", "host": _host()}


def run_reference_batched(args):
    """The oracle on a bounded sample of the 10,000-mesh batch: graphs/s of coarsening each
    sampled graph (3 levels) and its contraction gradient."""
    sub, one = _oracle_batch_sample()

    for _ in range(args.warmup):
        one()
    tot = sum(one() for _ in range(args.steps))
    value = sub.B * args.steps / tot
    line = {
        "impl": "reference", "metric": "batched fwd+bwd graphs/s", "value": value,
        "unit": "graphs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "c5_batch10k_f32", "sample_graphs": sub.B},
        "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sub.B} sampled graphs of the batch per step",
                         "host": _host()},
        "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    if args.workload == "c5_batch10k_f32":
        return run_reference_batched(args)
    spec = SAMPLES[args.workload]
    g = _sample_graph(spec)
    for _ in range(args.warmup):
        _oracle_step(g, spec)
    times, edges = [], 0
    for _ in range(args.steps):
        e, dt = _oracle_step(g, spec)
        edges += e
        times.append(dt)
    tot = sum(times)
    value = edges / tot / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": _dtype_of(spec),
        "data": "synthetic",
        "config": {"workload": args.workload, "sample_n": g.n, "sample_m": g.m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{spec.get('mode', 'halving')} coarsening of the reduced "
                                   f"construction (n={g.n}, m={g.m}) per step",
                         "host": _host()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _dtype_of(spec):
    return {"float64": "f64", "float32": "f32", "int32": "i32"}[spec["dtype"]]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# The binary64 score is bound by the FP64 pipe: its peak is the measured FP64 add rate of a
# GB300 (506.5 G additions/s, profiles/fp64_add_probe_gb300.md).
FP64_PEAK_GOPS = 506.5
FP64_PEAK_SOURCE = "measured FP64 add throughput (profiles/fp64_add_probe_gb300.md)"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a workload's dominant
# kernel, from single-pass ncu captures of the full-size workload (one step's launches summed
# and divided by the launches of a step, as `achieved` averages them; the commands and every
# launch are in profiles/traffic_dominant_kernels.md); absent where no capture of the current
# kernel exists (then `traffic` is null).
TRAFFIC = {
    ("c4_rgg8m_f32", "k_score_packed<Key>"): 2.236592e+09,
    ("c4_rgg8m_f32_one", "k_score_packed<Key>"): 1.393540e+10,
    ("c4_rgg8m_f32_reordered", "k_score_packed<Key>"): 4.090090e+08,
    ("c2_tri2048_f64", "(k_score_edges<P, Key, kScoreChains>)"): 2.226063e8,
    ("c3_tet129_f64", "(k_score_edges<P, Key, kScoreChains>)"): 3.163520e8,
    ("c5_batch10k_f32", "k_score_packed<Key>"): 3.834753e+09,
}

HEADLINE = "c4_rgg8m_f32"
# the other configurations reported in the same line (their own keys, fewer steps)
EXTRAS = ["c4_rgg8m_f32_one", "c4_rgg8m_f32_reordered", "c2_tri2048_f64", "c3_tet129_f64",
          "c5_batch10k_f32"]
# workloads run with the adjacency-reordering option
REORDERED = {"c4_rgg8m_f32_reordered"}


def _peaks():
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback (6.8 TB/s)"


def _roofline(workload, dominant, prof_entry, launches, ms, fp64):
    """Roofline of the dominant kernel from its timed launches: algorithmic bytes (the library's
    per-launch byte model: every input the operation needs read once, every output written
    once) or, for the binary64 score, the additions and subtractions it needs, over the
    launches' summed CUDA-event time."""
    hbm, src = _peaks()
    nbytes, ops = prof_entry[2], prof_entry[3]
    ach = nbytes / (ms * 1e-3) / 1e9 if nbytes > 0 and ms > 0 else None
    roof = {"kernel": dominant, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm if ach else None,
            "traffic": TRAFFIC.get((workload, dominant)), "peak_source": src,
            "launches": launches, "avg_launch_ms": ms / max(1, launches),
            "algorithmic_bytes_per_launch": nbytes / max(1, launches)}
    if ops > 0 and fp64:
        roof.update({"bound": "alu", "achieved": ops / (ms * 1e-3) / 1e9, "peak": FP64_PEAK_GOPS,
                     "unit": "G FP64 adds/s", "peak_source": FP64_PEAK_SOURCE,
                     "fp64_ops_per_launch": ops / max(1, launches),
                     "hbm_achieved_gbs": ach, "hbm_frac": ach / hbm if ach else None})
        roof["frac"] = roof["achieved"] / FP64_PEAK_GOPS
    return roof


def _dist_setup():
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    return ws, rank, local


def _max_over_ranks(t_ms, ws, dev):
    if ws == 1:
        return t_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


_GRAPHS = {}


def _config_graph(cfg_name):
    """The workload's graph, generated once per process (the one-level and the multilevel
    random geometric graph are the same graph)."""
    from paper_2204_11757_gb300 import inputs as I
    cfg = I.CONFIGS[cfg_name]
    key = tuple(sorted((k, str(v)) for k, v in cfg.items() if k not in ("mode", "ratio")))
    t0 = time.perf_counter()
    if key not in _GRAPHS:
        _GRAPHS.clear()
        _GRAPHS[key] = I.config_graph(cfg_name)[0]
    return _GRAPHS[key], cfg, time.perf_counter() - t0


def bench_single(workload, steps, warmup, e2e_on=True, pool=0, want_profile=False):
    """One step = one full coarsening of the workload (every level), inputs resident in HBM."""
    import torch
    import torch.distributed as dist
    from paper_2204_11757_gb300 import api
    ws, rank, local = _dist_setup()
    cfg_name, L, desc = WORKLOADS[workload]
    g, cfg, t_gen = _config_graph(cfg_name)
    n_c = max(1, g.n // cfg["ratio"])
    dev = torch.device("cuda", local)
    csr = api.CSR.from_graph(g, dev)
    ctx = api.Context(dev)
    stream = ctx.stream
    lift = torch.empty(g.n, dtype=torch.int32, device=dev)

    reorder = workload in REORDERED

    def step():
        ctx.coarsen(csr, n_c, levels=L, lift_out=lift, reorder=reorder)

    for _ in range(warmup):
        step()
    levels = [ctx.level_info(l) for l in range(ctx.level_count())]
    edges_per_step = sum(int(lv.m) for lv in levels)

    # one profiled step: per-kernel device time, to find the dominant kernel
    ctx.time_kernel("*")
    step()
    prof = ctx.kernel_profile()
    step_prof_ms = sum(v[1] for v in prof.values())
    dominant = max(prof.items(), key=lambda kv: kv[1][1])[0]

    # ---- timed region: the dominant kernel's launches carry CUDA events on the library's
    # stream (inside the captured graph) --------------------------------------------------------
    ctx.time_kernel(dominant)
    step()  # untimed: re-captures the schedule with the dominant kernel's events in it
    ctx.kernel_time()
    ctx.time_kernel(dominant)
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop() if rank == 0 else None
    launches = ctx.launch_count - launches0
    t_ms = _max_over_ranks(ev0.elapsed_time(ev1) / steps, ws, dev)
    dom_prof = ctx.kernel_profile()
    dom_launches, dom_ms = ctx.kernel_time()
    ctx.time_kernel(None)
    level_ms = [float(ctx.level_info(l).ms) for l in range(len(levels))]
    value = ws * edges_per_step / (t_ms * 1e-3) / 1e6
    roof = _roofline(workload, dominant, dom_prof.get(dominant, (0, 0.0, 0.0, 0.0)),
                     dom_launches, dom_ms, g.w.dtype != np.float32)

    # ---- end to end through host buffers: the pinned host CSR in, the lift and the final
    # coarse CSR out, every step ---------------------------------------------------------------
    e2e = None
    if e2e_on:
        host = api.CSR.from_graph(g, device="cpu", pin=True)
        lift_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
        bufs = None

        def e2e_step():
            nonlocal bufs
            ctx.coarsen(host, n_c, levels=L, lift_out=lift_h, reorder=reorder)
            info = ctx.level_info(ctx.level_count() - 1)
            if bufs is None or bufs[1].shape[0] < 2 * info.m_c:
                bufs = (torch.empty(info.n_c + 1, dtype=torch.int64).pin_memory(),
                        torch.empty(2 * info.m_c, dtype=torch.int32).pin_memory(),
                        torch.empty(2 * info.m_c, dtype=csr.w.dtype).pin_memory())
            for dst, src in zip(bufs, (info.rowptr_c, info.col_c, info.w_c)):
                ctx.lib.spc_copy(ctx._handle, api._ptr(dst), src, dst.numel() * dst.element_size())
            return info

        info = e2e_step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(1, min(steps, 5))
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ksteps):
            info = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = _max_over_ranks(e0.elapsed_time(e1) / ksteps, ws, dev)
        h2d = host.rowptr.numel() * 8 + host.col.numel() * 4 + host.w.numel() * host.w.element_size()
        d2h = g.n * 4 + (info.n_c + 1) * 8 + 2 * info.m_c * (4 + csr.w.element_size())
        e2e = {"value": ws * edges_per_step / (e_ms * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e_ms}

    # ---- node-feature pooling on the final lift (forward + backward), kernels timed live ------
    pooling = None
    if pool > 0:
        hbm, _ = _peaks()
        F = pool
        n_c_f = int(ctx.level_info(ctx.level_count() - 1).n_c)
        gen = torch.Generator(device=dev).manual_seed(0)
        x = torch.randn(g.n, F, dtype=torch.float32, device=dev, generator=gen)
        gxc = torch.randn(n_c_f, F, dtype=torch.float32, device=dev, generator=gen)
        for _ in range(2):
            ctx.pool_features(lift, n_c_f, x)
            ctx.pool_features_backward(lift, n_c_f, gxc)
        ctx.time_kernel("k_pool")
        reps = 5
        p0, p1, p2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        p0.record(stream)
        for _ in range(reps):
            ctx.pool_features(lift, n_c_f, x)
        p1.record(stream)
        for _ in range(reps):
            ctx.pool_features_backward(lift, n_c_f, gxc)
        p2.record(stream)
        torch.cuda.synchronize()
        kp = ctx.kernel_profile()
        ctx.time_kernel(None)
        top = max(kp.items(), key=lambda kv: kv[1][1])
        ach = top[1][2] / (top[1][1] * 1e-3) / 1e9 if top[1][2] > 0 else None
        pooling = {"features": F, "dtype": "f32", "n": g.n, "n_c": n_c_f,
                   "forward_ms": p0.elapsed_time(p1) / reps,
                   "backward_ms": p1.elapsed_time(p2) / reps,
                   "roofline": {"kernel": top[0], "bound": "hbm", "achieved": ach, "peak": hbm,
                                "unit": "GB/s", "frac": ach / hbm if ach else None}}
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": t_ms,
        "dtype": {np.dtype("float64"): "f64", np.dtype("float32"): "f32",
                  np.dtype("int32"): "i32"}[g.w.dtype],
        "config": {
            "workload": f"{workload}: {desc}", "n": g.n, "m": g.m, "n_c": n_c, "levels": L,
            "reorder": reorder,
            "multilevel_reading": "self-mass (the merged node of Theorem 2's proof)",
            "parallelism": "replicas" if ws > 1 else "single GPU",
            "l2": "inputs larger than L2 (%.0f MB resident CSR)" % (
                (csr.rowptr.numel() * 8 + csr.col.numel() * 4
                 + csr.w.numel() * csr.w.element_size()) / 1e6),
            "generation_s": round(t_gen, 1),
            "per_level": [{"n": int(lv.n), "m": int(lv.m), "n_c": int(lv.n_c),
                           "m_c": int(lv.m_c), "ms": ms,
                           "M_edges_s": (int(lv.m) / (ms * 1e-3) / 1e6) if ms > 0 else None}
                          for lv, ms in zip(levels, level_ms)],
        },
        "roofline": roof, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
        "steps": steps, "warmup": warmup,
    }
    if pooling is not None:
        res["pooling"] = pooling
    if want_profile:
        res["kernel_profile"] = {k: [v[0], round(v[1], 4)] for k, v in
                                 sorted(prof.items(), key=lambda kv: -kv[1][1])}
        res["profiled_step_ms"] = step_prof_ms
    ctx.close()
    del csr, lift
    torch.cuda.empty_cache()
    return res


def bench_batched(steps, warmup, want_profile=False, cpu=False):
    """Batched forward + backward: one coarsening of every graph of the batch (3 halving levels,
    one set of launches for all graphs), the coarse weights through the differentiable
    contraction, loss sum(a * g), backward to the fine weights.  graphs/s = B / step time,
    against a loop that coarsens the graphs one by one with the single-graph entry point."""
    import torch
    import torch.distributed as dist
    from paper_2204_11757_gb300 import api, inputs as I, shard as S

    ws, rank, local = _dist_setup()
    t_gen = time.perf_counter()
    full, cfg = I.config_graph("c5_batch10k_f32")
    t_gen = time.perf_counter() - t_gen
    batch, (g0, g1) = S.local_batch(full, rank, ws) if ws > 1 else (full, (0, full.B))
    dev = torch.device("cuda", local)
    csr = api.CSR.from_graph(batch.graph, dev)
    gptr = torch.from_numpy(batch.graph_ptr).to(dev)
    w_und = torch.from_numpy(batch.graph.w_und).to(dev)
    ctx = api.Context(dev)
    L = 3

    def step():
        ctx.coarsen_batched(csr, gptr, cfg["ratio"], L)
        plan = api.ContractionPlan.from_levels(ctx, ctx.levels())
        w = w_und.detach().requires_grad_(True)
        a = api.contract_weights(w, plan)
        gvec = torch.ones_like(a)
        (a * gvec).sum().backward()
        return w.grad

    for _ in range(warmup):
        step()
    # one profiled step finds the dominant kernel; the timed steps time its launches
    ctx.time_kernel("*")
    step()
    prof = ctx.kernel_profile()
    dominant = max(prof.items(), key=lambda kv: kv[1][1])[0]
    ctx.time_kernel(dominant)
    step()  # untimed: re-captures with the dominant kernel's events
    ctx.kernel_time()
    ctx.time_kernel(dominant)
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(ctx.stream)
    for _ in range(steps):
        step()
    ev1.record(ctx.stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if rank == 0 else None
    t_ms = _max_over_ranks(ev0.elapsed_time(ev1) / steps, ws, dev)
    launches = ctx.launch_count - launches0
    dom_prof = ctx.kernel_profile()
    dom_launches, dom_ms = ctx.kernel_time()
    ctx.time_kernel(None)
    roof = _roofline("c5_batch10k_f32", dominant, dom_prof.get(dominant, (0, 0.0, 0.0, 0.0)),
                     dom_launches, dom_ms, False)

    # end to end: the batch in pinned host memory, copied in by the library; the gradient
    # of the fine weights and the per-graph coarse offsets read back
    host = api.CSR.from_graph(batch.graph, device="cpu", pin=True)
    gptr_h = torch.from_numpy(batch.graph_ptr).pin_memory()
    grad_h = torch.empty(batch.graph.m, dtype=torch.float32).pin_memory()
    w_h = torch.from_numpy(batch.graph.w_und).pin_memory()

    ranges = S.shard_ranges(S.batch_edge_counts(full), ws) if ws > 1 else None

    def gather_counts(parts, t):
        # NCCL gathers device tensors; global_offsets hands host ones
        dparts = [torch.empty_like(t, device=dev) for _ in parts]
        dist.all_gather(dparts, t.to(dev))
        for p, d in zip(parts, dparts):
            p.copy_(d.cpu())

    def e2e_step():
        _, gpc, _ = ctx.coarsen_batched(host, gptr_h, cfg["ratio"], L)
        plan = api.ContractionPlan.from_levels(ctx, ctx.levels())
        w = w_h.to(dev, non_blocking=True)
        w.requires_grad_(True)
        a = api.contract_weights(w, plan)
        (a * torch.ones_like(a)).sum().backward()
        grad_h.copy_(w.grad, non_blocking=True)
        if ranges is not None:
            # the one collective of a sharded batch: every rank's per-graph super-node
            # counts, for the global offsets of the coarse graphs
            counts = torch.diff(gpc.cpu()).numpy()
            return S.global_offsets(counts, ranges, ws, all_gather=gather_counts)
        return gpc

    e2e_step()
    torch.cuda.synchronize()
    k = max(1, min(steps, 3))
    t0 = time.perf_counter()
    for _ in range(k):
        e2e_step()
    torch.cuda.synchronize()
    e_ms = _max_over_ranks((time.perf_counter() - t0) * 1e3 / k, ws, dev)
    h2d = (host.rowptr.numel() * 8 + host.col.numel() * 4 + host.w.numel() * 4
           + gptr_h.numel() * 8 + batch.graph.m * 4)
    d2h = batch.graph.m * 4 + (batch.B + 1) * 8 + batch.graph.n * 4
    e2e = {"value": ws * batch.B / (e_ms * 1e-3), "unit": "graphs/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": e_ms}
    value = full.B / (t_ms * 1e-3)
    # per-graph loop of the single-graph coarsener on a sample, same work per graph
    loop = None
    if rank == 0:
        rng = np.random.default_rng(0)
        idx = np.sort(rng.choice(batch.B, size=min(100, batch.B), replace=False))
        subs = [I.subsample_batch(batch, [i]) for i in idx]
        gs = [(api.CSR.from_graph(s.graph, dev), torch.from_numpy(s.graph.w_und).to(dev),
               s.graph.n) for s in subs]

        def one(gc, wu, n):
            ctx.coarsen(gc, max(1, n // cfg["ratio"]), levels=L)
            plan = api.ContractionPlan.from_levels(ctx, ctx.levels())
            w = wu.detach().requires_grad_(True)
            a = api.contract_weights(w, plan)
            (a * torch.ones_like(a)).sum().backward()

        for gc, wu, n in gs[:5]:
            one(gc, wu, n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for gc, wu, n in gs:
            one(gc, wu, n)
        torch.cuda.synchronize()
        loop_s = (time.perf_counter() - t0) / len(gs)
        loop = {"graphs_s": 1.0 / loop_s, "sample_graphs": len(gs),
                "what": "the same forward + backward, graph by graph, through spc_coarsen"}
    res = {
        "metric": "batched fwd+bwd graphs/s", "value": value, "unit": "graphs/s",
        "ms_per_step": t_ms, "dtype": "f32", "steps": steps, "warmup": warmup,
        "config": {"workload": "c5_batch10k_f32: 10,000 jittered 2D/3D meshes, node counts "
                               "log-uniform 200-20,000, FP32 1/edge-length, 3 halving "
                               "levels to n_b/8 each, forward + backward through the "
                               "contraction", "B": full.B, "n": full.graph.n,
                   "m": full.graph.m, "parallelism": f"graphs sharded over {ws} rank(s)",
                   "generation_s": round(t_gen, 1), "per_graph_loop": loop,
                   "speedup_vs_per_graph_loop": (value / loop["graphs_s"]) if loop else None},
        "roofline": roof, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
        "cpu_baseline": _oracle_batched() if (cpu and ws == 1 and rank == 0) else None,
    }
    if want_profile:
        res["kernel_profile"] = {k: [v[0], round(v[1], 4)] for k, v in
                                 sorted(prof.items(), key=lambda kv: -kv[1][1])}
    ctx.close()
    del csr, gptr, w_und
    torch.cuda.empty_cache()
    return res


def _summary(res):
    """The keys of an extra configuration kept in the headline's line."""
    keep = ("metric", "value", "unit", "ms_per_step", "dtype", "roofline", "e2e", "clocks",
            "gpu_launches", "steps", "warmup", "kernel_profile")
    out = {k: res[k] for k in keep if k in res}
    cfg = dict(res["config"])
    out["config"] = cfg
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["c5_batch10k_f32"],
                    default=HEADLINE)
    ap.add_argument("--no-extras", action="store_true",
                    help="only the chosen workload (default: the headline adds the other "
                         "configurations as keys of the same line)")
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="print the per-kernel breakdown")
    ap.add_argument("--pool", type=int, default=64,
                    help="also time node-feature pooling of this many binary32 features on the "
                         "final lift (0: off)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import __graft_entry__ as ge
    ws, rank, local = _dist_setup()
    if rank == 0:
        ge.build()
    if ws > 1:
        dist.barrier()

    if args.workload == "c5_batch10k_f32":
        res = bench_batched(args.steps, args.warmup, args.profile, not args.no_cpu_baseline)
    else:
        res = bench_single(args.workload, args.steps, args.warmup, not args.no_e2e, args.pool,
                           args.profile)
        res["cpu_baseline"] = (cpu_baseline(args.workload) if rank == 0 and ws == 1
                               and not args.no_cpu_baseline else None)
    extras = {}
    if args.workload == HEADLINE and not args.no_extras:
        for name in EXTRAS:
            st = max(1, args.extra_steps)
            if name == "c5_batch10k_f32":
                r = bench_batched(st, args.warmup, args.profile)
            else:
                r = bench_single(name, st, args.warmup, e2e_on=False, pool=0,
                                 want_profile=args.profile)
            extras[name] = _summary(r)
    if rank == 0:
        line = {
            "metric": res["metric"], "value": res["value"], "unit": res["unit"], "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True,
            "scaling": "strong" if args.workload == "c5_batch10k_f32" else "weak",
            "vs_baseline": None, "dtype": res["dtype"], "data": "synthetic",
            "config": res["config"], "roofline": res["roofline"],
            "cpu_baseline": res.get("cpu_baseline"), "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": res["gpu_launches"],
        }
        for k in ("pooling", "kernel_profile", "profiled_step_ms"):
            if k in res:
                line[k] = res[k]
        if extras:
            line["configs"] = extras
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
