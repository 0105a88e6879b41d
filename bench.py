#!/usr/bin/env python
"""Benchmark: Barnes-Hut bodies/s per leapfrog step on one GB300.

Workload (default): two colliding Plummer spheres of 8,388,608 equal-mass bodies each
(N = 16,777,216, G = 1, total mass 1, centres at x = -5 and +5, closing speed 0.5), softening
eps = 0.002, opening angle theta = 0.5, dt = 5e-4, FP32 forces with compensated (Kahan)
accumulation and FP64 positions and velocities.  A step is one full kick-drift-kick step through
the C ABI (nbody_step): kick + drift + root box, Morton keys, radix sort, permutation, node
split, moments, walk + second kick.  Inputs (0.94 GB) are larger than L2 (129 MB), so no flush
is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own independent replica (no collective on the
data path): value = all ranks' bodies / max-over-ranks time.  `--impl reference` times the CPU
oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ics  # noqa: E402

METRIC = "Barnes-Hut bodies/s per step at N=16M θ=0.5 (FP32 vs FP64); batch steps/s"
FLOP_PER_INTERACTION = 20          # softened monopole pair term, counting rsqrt as 2 flops
FP32_LANES_PER_SM = 128            # FP32 FMA lanes per SM (Blackwell)
# Algorithmic bytes per body of the build phases (compulsory reads + writes):
#   kick + drift + box partials: pos, vel, acc, mass read (80 B), pos, vel written (48 B), the
#   (x, y, z, m) record for the permutation written (32 B); keys: pos read (24 B), key + id
#   written (12 B)
BYTES_KICK_KEYS = 80 + 48 + 32 + 24 + 12
#   radix sort: digit histograms read the keys once (8 B); each of 8 passes reads the keys in the
#   upsweep (8 B) and reads + writes keys and ids in the downsweep (24 B)
BYTES_SORT = 8 + 8 * (8 + 24)
# Re-sort from the previous order (§4.4) instead of keys + radix sort:
#   extract: previous id read (4 B), the body's (x, y, z, m) record gathered (32 B), key written
#   (8 B)
BYTES_KICK_EXTRACT = 80 + 48 + 32 + 4 + 32 + 8
#   split: key + id read, written to the kept or removed list (24 B); merge: both lists read,
#   keys + ids written (24 B); plus, per removed body, the radix sort by (key, id) with 3 id
#   passes (8 + 11 * 32 B)
BYTES_RESORT_FIXED = 24 + 24
BYTES_RESORT_PER_REMOVED = 8 + 11 * 32
CPU_SAMPLE_N = 1 << 20             # bodies in the CPU-baseline sample
CPU_SAMPLE_STEPS = 3               # timed oracle steps on that sample (about 10-15 s on 16 cores)
REF_SAMPLE_N = 1 << 20             # bodies per step of the reference arm


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="two_plummer_16m", choices=sorted(ics.WORKLOADS))
    ap.add_argument("--n", "--bodies", dest="n", type=int, default=0,
                    help="override N (smaller runs, profiling; --bodies under torchrun)")
    ap.add_argument("--precision", default="fp32_kahan", choices=["fp64", "fp32", "fp32_kahan"])
    ap.add_argument("--theta", type=float, default=None)
    ap.add_argument("--sort", default="auto", choices=["auto", "full"],
                    help="auto: re-sort from the previous step's order (§4.4); full: radix sort")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-system forest line")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the per-theta error report")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 step on the same workload (the FP64 side of the metric)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the 512-system forest (FP32-Kahan), one JSON line with its figures")
    ap.add_argument("--batch-steps", type=int, default=100, help="graph-replayed forest steps")
    ap.add_argument("--walk-shape", type=int, default=None,
                    help="use this walk launch shape instead of the autotuner's choice (profiling "
                         "runs: the autotuner's timings are not meaningful under a profiler)")
    return ap.parse_args()


def make_workload(name, n_override=0):
    w = dict(ics.WORKLOADS[name])
    n = n_override or w["n"]
    if w["kind"] == "two_plummer":
        pos, vel, mass = ics.two_plummer(n, seeds=w["seeds"])
    elif w["kind"] == "plummer":
        pos, vel, mass = ics.plummer(n, w["seed"])
    elif w["kind"] == "disk_bulge":
        pos, vel, mass = ics.disk_bulge(n, w["seed"])
    else:
        raise SystemExit(f"workload {name} is not a single system")
    w["n"] = n
    return w, pos, vel, mass


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle (baseline only)

def oracle_step_rate(name, w, n_sample, steps=1):
    """Bodies/s per step of the CPU oracle (FP64 Barnes-Hut + KDK) on `n_sample` bodies drawn
    with the same recipe as the workload; OpenMP over all host cores for the force walk."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    _, pos, vel, mass = make_workload(name, n_sample)
    acc, _, _ = oracle.bh(pos, mass, 1.0, w["eps"], w["theta"])
    t0 = time.perf_counter()
    oracle.kdk(pos, vel, mass, acc, 1.0, w["eps"], w["theta"], w["dt"], steps)
    dt = time.perf_counter() - t0
    return n_sample * steps / dt, dt, cores


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.destroy_process_group()
            return
    w = dict(ics.WORKLOADS[args.workload])
    if args.theta is not None:
        w["theta"] = args.theta
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    sample_n = args.n or REF_SAMPLE_N
    _, pos, vel, mass = make_workload(args.workload, sample_n)
    acc, _, _ = oracle.bh(pos, mass, 1.0, w["eps"], w["theta"])
    for _ in range(args.warmup):
        pos, vel, acc = oracle.kdk(pos, vel, mass, acc, 1.0, w["eps"], w["theta"], w["dt"], 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pos, vel, acc = oracle.kdk(pos, vel, mass, acc, 1.0, w["eps"], w["theta"], w["dt"], 1)
    dt = time.perf_counter() - t0
    value = sample_n * args.steps / dt
    sample = (f"CPU oracle (FP64 pointer-octree Barnes-Hut by insertion + KDK), "
              f"{sample_n} bodies drawn with the workload's recipe per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "bodies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} sampled at N={sample_n}",
                   "theta": w["theta"], "eps": w["eps"], "dt": w["dt"]},
        "cpu_baseline": {"value": value, "unit": "bodies/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "bodies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ GPU arm

def measure_batch(nb, torch, dev, stream, steps=100, with_fp64=True):
    """The batched forest (512 Plummer systems, N_s log-uniform in [1024, 65536], eps 0.01,
    theta 0.6, dt 1e-3, FP32-Kahan forces): `steps` leapfrog steps replayed from one captured
    CUDA graph, timed with CUDA events on the context stream; plus the same steps launched
    kernel by kernel for comparison."""
    w = ics.WORKLOADS["forest_512"]
    pos, vel, mass, off = ics.forest(w["systems"], w["seed"])
    n = int(off[-1])
    tp = torch.from_numpy(pos).to(dev)
    tv = torch.from_numpy(vel).to(dev)
    tm = torch.from_numpy(mass).to(dev)
    ctx = nb.Context.forest(off, 1.0, w["eps"], w["theta"], w["dt"], nb.FP32_KAHAN, stream=stream)
    shape, shape_ms = ctx.autotune(tp, tm)
    shape_threads = ctx.walk_shape()[1]
    ctx.forest_step(tp, tv, tm, 4, use_graph=True)     # a^(0), capture, warm-up replays
    ctx.forest_step(tp, tv, tm, 3, use_graph=False)    # warm-up of the launched form
    ctx.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    l0 = nb.launch_count()
    ev[0].record(stream)
    ctx.forest_step(tp, tv, tm, steps, use_graph=True)
    ev[1].record(stream)
    torch.cuda.synchronize()
    launches = nb.launch_count() - l0
    k = max(1, steps // 10)
    ev[2].record(stream)
    ctx.forest_step(tp, tv, tm, k, use_graph=False)
    ev[3].record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    # the walk of one force evaluation of the same forest: its useful FP32 rate (outside the
    # timed region), against the FP32 peak of the main line
    ctx.enable_timing(True)
    acc = ctx.forest_forces(tp, tm)
    acc = ctx.forest_forces(tp, tm, acc)
    walk_ms = float(ctx.timings()[3])
    pp, pc = ctx.counters(n)
    ctx.enable_timing(False)
    inter = float(pp.astype(np.float64).sum() + pc.astype(np.float64).sum())
    peaks, _ = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tf = sms * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    tf = inter * FLOP_PER_INTERACTION / (walk_ms * 1e-3) / 1e12
    ctx.close()
    ms = ev[0].elapsed_time(ev[1])
    ms_launched = ev[2].elapsed_time(ev[3]) / k
    # the plain FP64 path on the same forest, one launched step after its starting forces
    ms64 = None
    if with_fp64:
        with nb.Context.forest(off, 1.0, w["eps"], w["theta"], w["dt"], nb.FP64,
                               stream=stream) as c64:
            c64.forest_step(tp, tv, tm, 1, use_graph=False)
            c64.sync()
            ev[0].record(stream)
            c64.forest_step(tp, tv, tm, 1, use_graph=False)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms64 = ev[0].elapsed_time(ev[1])
    return {"metric": "batch steps/s", "value": steps / (ms * 1e-3), "unit": "steps/s",
            "workload": "forest_512", "systems": int(w["systems"]), "bodies": n,
            "bodies_per_s": n * steps / (ms * 1e-3), "ms_per_step": ms / steps,
            "ms_per_step_launched": ms_launched, "ms_per_step_fp64": ms64,
            "steps": steps, "graph": True,
            "gpu_launches": int(launches), "precision": "fp32_kahan",
            "walk_shape": {"chosen": shape, "threads_per_block": shape_threads,
                           "autotune_ms": shape_ms},
            "walk": {"ms": walk_ms, "interactions": inter, "achieved_tflops": tf,
                     "peak_tflops": peak_tf, "frac": tf / peak_tf, "bound": "alu"},
            "theta": w["theta"], "eps": w["eps"], "dt": w["dt"]}


def measure_accuracy(nb, torch, dev, stream, n_targets=16384):
    """Force errors on the 1,048,576-body Plummer sphere (eps 0.005) against the FP64 direct
    sum on 16,384 sampled targets, per theta, for the plain FP64 path, the FP32-Kahan path and
    the FP32-Kahan path with the grouped acceptance test (NBODY_FLAG_GROUP_MAC) or with
    quadrupole cell terms (NBODY_FLAG_QUADRUPOLE), with the walk time of each on this GPU.""" 
    w = ics.WORKLOADS["plummer_1m"]
    pos, _, mass = ics.plummer(w["n"], w["seed"])
    n = w["n"]
    tp = torch.from_numpy(pos).to(dev)
    tm = torch.from_numpy(mass).to(dev)
    rng = np.random.Generator(np.random.PCG64(3))
    tgt = np.sort(rng.choice(n, n_targets, replace=False)).astype(np.int64)
    tt = torch.from_numpy(tgt).to(dev)

    def rel(a, ref):
        num = ((a - ref) ** 2).sum(axis=0)
        den = (ref ** 2).sum(axis=0)
        return {"rms": float(np.sqrt(np.mean(num / den))),
                "global": float(np.sqrt(num.sum() / den.sum())),
                "p99": float(np.sqrt(np.quantile(num / den, 0.99)))}

    direct_rate = {}
    fp64_peak = nb.measure_fp64_rate(stream)
    fp32_peak = nb.measure_fp32_rate(stream)
    for name, prec in (("fp64", nb.FP64), ("fp64_fast", nb.FP64_FAST), ("fp32", nb.FP32)):
        with nb.Context(n, 1.0, w["eps"], 0.5, w["dt"], prec, stream=stream) as ctx:
            a = ctx.direct_forces(tp, tm, tt)   # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            a = ctx.direct_forces(tp, tm, tt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            pairs = float(n_targets) * (n - 1)
            tf = pairs * FLOP_PER_INTERACTION / (ms * 1e-3) / 1e12
            peak = fp32_peak if name == "fp32" else fp64_peak
            direct_rate[name] = {"ms": ms, "pairs": pairs, "tflops": tf,
                                 "frac_of_fma_probe": tf / peak if peak > 0 else None}
            if name == "fp64":
                direct = a.cpu().numpy()
    out = {"workload": "plummer_1m", "n": n, "eps": w["eps"], "targets": n_targets,
           "reference": "FP64 direct sum (nbody_direct_forces) on the sampled targets",
           "direct_sum": direct_rate, "theta": {}}
    for theta in (0.3, 0.5, 0.7):
        row = {}
        res = {}
        for name, prec, flags in (("fp64", nb.FP64, 0), ("fp64_fast", nb.FP64_FAST, 0),
                                  ("fp32", nb.FP32, 0), ("fp32_kahan", nb.FP32_KAHAN, 0),
                                  ("fp32_kahan_group_mac", nb.FP32_KAHAN, nb.FLAG_GROUP_MAC),
                                  ("fp32_kahan_quadrupole", nb.FP32_KAHAN, nb.FLAG_QUADRUPOLE)):
            with nb.Context(n, 1.0, w["eps"], theta, w["dt"], prec, stream=stream,
                            flags=flags) as ctx:
                ctx.autotune(tp, tm)
                ctx.enable_timing(True)
                a = ctx.forces(tp, tm)
                t = ctx.timings()
                a = a.cpu().numpy()
                pp, pc = ctx.counters(n)
            res[name] = a
            row[name] = {"vs_direct": rel(a[:, tgt], direct), "walk_ms": float(t[3]),
                         "interactions_per_body": float((pp.astype(np.float64).sum() +
                                                         pc.astype(np.float64).sum()) / n)}
        row["fp32_kahan_vs_fp64_bh"] = rel(res["fp32_kahan"], res["fp64"])
        row["fp32_vs_fp64_bh"] = rel(res["fp32"], res["fp64"])
        row["fp64_fast_vs_fp64_bh"] = rel(res["fp64_fast"], res["fp64"])
        out["theta"][str(theta)] = row
    out["energy"] = measure_energy_drift(nb, torch, dev, stream)
    return out


def plain_energy(pos, vel, mass, eps):
    """Total energy E_kin + E_pot (§2.3: softened pair potential summed over i < j, G = 1) of a
    host state, a plain numpy pair sum written for this report."""
    pos = np.asarray(pos, np.float64)
    vel = np.asarray(vel, np.float64)
    mass = np.asarray(mass, np.float64)
    ekin = 0.5 * float(np.sum(mass * np.sum(vel * vel, axis=0)))
    epot = 0.0
    n = mass.shape[0]
    for i in range(n - 1):
        d = pos[:, i + 1:] - pos[:, i:i + 1]
        r = np.sqrt(np.sum(d * d, axis=0) + eps * eps)
        epot -= mass[i] * float(np.sum(mass[i + 1:] / r))
    return ekin + epot


def measure_energy_drift(nb, torch, dev, stream):
    """Relative energy drift (E_10 - E_0) / |E_0| and momentum change of 10 KDK steps on the
    4096-body Plummer configuration (eps 0.01, theta 0.5, dt 1e-3) for every precision form."""
    w = ics.WORKLOADS["plummer_4k"]
    pos, vel, mass = ics.plummer(w["n"], w["seed"])
    e0 = plain_energy(pos, vel, mass, w["eps"])
    p0 = (vel * mass[None, :]).sum(axis=1)
    out = {"workload": "plummer_4k", "steps": w["steps"], "dt": w["dt"],
           "energy": "plain numpy pair sum over i < j"}
    for name, prec in (("fp64", nb.FP64), ("fp64_fast", nb.FP64_FAST), ("fp32", nb.FP32),
                       ("fp32_kahan", nb.FP32_KAHAN)):
        tp, tv = torch.from_numpy(pos).to(dev), torch.from_numpy(vel).to(dev)
        with nb.Context(w["n"], 1.0, w["eps"], w["theta"], w["dt"], prec, stream=stream) as ctx:
            ctx.step(tp, tv, torch.from_numpy(mass).to(dev), w["steps"])
            ctx.sync()
        p, v = tp.cpu().numpy(), tv.cpu().numpy()
        out[name] = {"drift": (plain_energy(p, v, mass, w["eps"]) - e0) / abs(e0),
                     "dP": float(np.linalg.norm((v * mass[None, :]).sum(axis=1) - p0))}
    return out


# the walk kernel's source: its DRAM traffic from the committed capture is reported only while
# this file is unchanged
WALK_SOURCES = ("paper_2203_08966_gb300/csrc/walk_kernels.cu",)
WALK_PROFILE = "profiles/pb_walk32_two_plummer_16m.md"


def walk_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in WALK_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def committed_traffic():
    """DRAM bytes per walk launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
    committed ncu summary of the benchmark workload, or None when that summary is missing or
    was taken on other walk sources than the ones built now."""
    try:
        with open(os.path.join(ROOT, WALK_PROFILE)) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        line = line.strip().strip("`")
        for key in ("traffic_bytes_per_launch:", "walk_sources_sha256:"):
            if line.startswith(key):
                vals[key] = line[len(key):].strip()
    if vals.get("walk_sources_sha256:") != walk_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch:"])
    except (KeyError, ValueError):
        return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    import paper_2203_08966_gb300 as nb

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    nb.load_library()
    if args.batch_only:
        if rank == 0:
            dev = torch.device("cuda", local)
            b = measure_batch(nb, torch, dev, torch.cuda.current_stream(), args.batch_steps,
                              with_fp64=False)
            print(json.dumps({"batch": b}))
        if ws > 1:
            dist.destroy_process_group()
        return

    w, pos, vel, mass = make_workload(args.workload, args.n)
    if args.theta is not None:
        w["theta"] = args.theta
    n = w["n"]
    prec = nb.PRECISIONS[args.precision]
    dev = torch.device("cuda", local)
    tp = torch.from_numpy(pos).to(dev)
    tv = torch.from_numpy(vel).to(dev)
    tm = torch.from_numpy(mass).to(dev)
    stream = torch.cuda.current_stream()

    ctx = nb.Context(n, 1.0, w["eps"], w["theta"], w["dt"], prec, stream=stream)
    ctx.set_sort_mode(nb.SORT_FULL if args.sort == "full" else nb.SORT_AUTO)
    if args.walk_shape is None:
        shape, shape_ms = ctx.autotune(tp, tm)   # launch shape of the walk, before any timing
    else:
        ctx.set_walk_shape(args.walk_shape)
        shape, shape_ms = args.walk_shape, None
    shape_threads = ctx.walk_shape()[1]
    ctx.enable_timing(True)
    for _ in range(args.warmup):
        ctx.step(tp, tv, tm, 1)
    ctx.sync()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    walk_ms, phase = [], np.zeros(5)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = nb.launch_count()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.step(tp, tv, tm, 1)
            t = ctx.timings()
            walk_ms.append(float(t[3]))
            phase += t
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = nb.launch_count() - l0
    sort_path, sort_removed = ctx.sort_stats()   # of the last timed step
    # measured FP32 FMA rate of this GPU (outside the timed region): the walk's fraction of it
    ffma_tflops = nb.measure_fp32_rate(stream)
    if sort_path == 1:
        b_keys = BYTES_KICK_EXTRACT
        b_sort = BYTES_RESORT_FIXED + BYTES_RESORT_PER_REMOVED * sort_removed / n
    else:
        b_keys, b_sort = BYTES_KICK_KEYS, BYTES_SORT
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    t_max = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms_max = float(t_max.item())
    value = n * ws * args.steps / (ms_max * 1e-3)

    # interactions of the last timed step (counters of its walk) -> algorithmic FP32 flops
    pp, pc = ctx.counters(n)
    inter = float(pp.astype(np.float64).sum() + pc.astype(np.float64).sum())
    walk_avg = float(np.mean(walk_ms))
    achieved = inter * FLOP_PER_INTERACTION / (walk_avg * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, peak_src = load_peaks()
    clk = clocks.summary()
    peak_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tf = sms * FP32_LANES_PER_SM * 2 * peak_mhz * 1e6 / 1e12

    # the FP64 side of the metric: one step of each FP64 form on the same workload (after its
    # starting forces and one warm-up step), CUDA events on the context stream, with the walk's
    # useful FP64 rate against the measured FP64 FMA rate
    fp64 = None
    if ws == 1 and not args.no_fp64:
        fp64_peak = nb.measure_fp64_rate(stream)
        fp64 = {"fp64_fma_probe_tflops": fp64_peak,
                "fp64_peak_source": "nbody_measure_fp64_rate: independent FP64 FMA chains on "
                                    "every SM, CUDA events"}
        for name, prec in (("fp64", nb.FP64), ("fp64_fast", nb.FP64_FAST)):
            p64, v64 = torch.from_numpy(pos).to(dev), torch.from_numpy(vel).to(dev)
            with nb.Context(n, 1.0, w["eps"], w["theta"], w["dt"], prec, stream=stream) as c64:
                c64.step(p64, v64, tm, 1)
                c64.sync()
                c64.enable_timing(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                c64.step(p64, v64, tm, 1)
                e1.record(stream)
                torch.cuda.synchronize()
                ms64 = e0.elapsed_time(e1)
                wms = float(c64.timings()[3])
                pp64, pc64 = c64.counters(n)
            del p64, v64
            i64 = float(pp64.astype(np.float64).sum() + pc64.astype(np.float64).sum())
            ach = i64 * FLOP_PER_INTERACTION / (wms * 1e-3) / 1e12
            fp64[name] = {"value": n / (ms64 * 1e-3), "unit": "bodies/s", "ms_per_step": ms64,
                          "walk_ms": wms, "interactions": i64,
                          "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak,
                                       "unit": "TFLOP/s", "frac": ach / fp64_peak if
                                       fp64_peak > 0 else None}}
        fp64["note"] = ("fp64: the bit-exact FP64 path (every pair term separately rounded, "
                        "correctly rounded square root and division, the oracle's order); "
                        "fp64_fast: the same FP64 acceptance test and interaction lists, pair "
                        "terms with fused multiply-adds and one rsqrt.  FP32-Kahan over FP64 = "
                        "value / fp64_fast.value (the faster FP64 form)")

    batch = None
    accuracy = None
    if ws == 1 and not args.no_batch:
        batch = measure_batch(nb, torch, dev, stream)
    if ws == 1 and not args.no_accuracy:
        accuracy = measure_accuracy(nb, torch, dev, stream)

    # end to end through the host-buffer entry point: pinned inputs copied in, result read back
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(pos).pin_memory().numpy()
        hv = torch.from_numpy(vel).pin_memory().numpy()
        hm = torch.from_numpy(mass).pin_memory().numpy()
        ctx.enable_timing(False)
        # a^(0) at the initial positions (set-up, outside the timed region)
        ha = ctx.forces(torch.from_numpy(pos).to(dev), tm).cpu().pin_memory().numpy()
        ctx.step_host(hp, hv, hm, 1, acc=ha)    # warm-up of the host path
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.step_host(hp, hv, hm, 1, acc=ha)
        e2e_s = time.perf_counter() - t0
        t_e = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
        e2e = {"value": n * ws * args.steps / float(t_e.item()), "unit": "bodies/s",
               "h2d_bytes_per_step": int(hp.nbytes + hv.nbytes + ha.nbytes + hm.nbytes),
               "d2h_bytes_per_step": int(hp.nbytes + hv.nbytes + ha.nbytes),
               "api": "nbody_step_host (pinned host buffers, one step per call)"}
    ctx.close()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        rate, secs, cores = oracle_step_rate(args.workload, w, CPU_SAMPLE_N, CPU_SAMPLE_STEPS)
        cpu = {"value": rate, "unit": "bodies/s", "cores": cores, "kind": "oracle",
               "sample": f"{CPU_SAMPLE_STEPS} KDK steps of the FP64 CPU oracle on {CPU_SAMPLE_N} "
                         f"bodies drawn with the same recipe ({secs:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": "bodies/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "fp32_kahan": "f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload if not args.n else
                   f"{args.workload} recipe at n = {n}", "n": n, "theta": w["theta"], "eps": w["eps"],
                   "dt": w["dt"], "precision": args.precision,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{ws}",
                   "walk_shape": {"chosen": shape, "threads_per_block": shape_threads,
                                  "autotune_ms": shape_ms}},
        "phase_ms": {k: float(v / args.steps) for k, v in
                     zip(("kick_box_keys", "sort", "permute_split_moments", "walk", "step"),
                         phase)},
        "sort": {"mode": args.sort, "path": "resort" if sort_path == 1 else "full",
                 "removed_fraction": (sort_removed / n) if sort_removed >= 0 else None},
        "build_roofline": {
            "unit": "GB/s", "peak": peaks.get("hbm_gbs"), "peak_source": f"{peak_src} copy bandwidth",
            "kick_box_keys": {"bytes_per_body": b_keys,
                              "achieved": b_keys * n / (phase[0] / args.steps * 1e-3) / 1e9},
            "sort": {"bytes_per_body": b_sort,
                     "achieved": b_sort * n / (phase[1] / args.steps * 1e-3) / 1e9}},
        "interactions_per_step": inter,
        "interactions_per_s": inter / (walk_avg * 1e-3),
        "roofline": {"kernel": "walk32 (Kahan)" if args.precision == "fp32_kahan" else
                     ("walk32" if args.precision == "fp32" else "walk64"),
                     "bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf,
                     "traffic": committed_traffic() if args.precision == "fp32_kahan" and
                     args.workload == "two_plummer_16m" and not args.n else None,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + "
                                     "dram__bytes_write.sum)",
                     "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                    f"{peak_mhz:.0f} MHz ({peak_src} max SM clock)",
                     "ffma_probe": {"tflops": ffma_tflops, "frac": achieved / ffma_tflops
                                    if ffma_tflops > 0 else None,
                                    "source": "nbody_measure_fp32_rate: independent FP32 FMA "
                                              "chains on every SM, CUDA events"},
                     "walk_ms": walk_avg},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fp64": fp64,
        "batch": batch,
        "accuracy": accuracy,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
