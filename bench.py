#!/usr/bin/env python
"""Benchmark: FP64 numeric refactorization + solve of the 200k-unknown
synthetic power-grid matrix (400x500 mesh, 64 supply nets, 2% controlled
sources, nested-dissection order), one Newton-style step = new values ->
glu_factor -> glu_solve (1 right-hand side).

Prints one JSON line.  ``--impl reference`` times the CPU oracle (plain
Gilbert-Peierls LU + solves) on the same workload instead.  Under torchrun
every rank runs an independent replica on its own GPU (a single
factorization does not shard); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "mesh400x500_nets64"
VALUE_SEEDS = list(range(1001, 1011))      # ten re-drawn value sets
METRIC = "FP64 numeric refactor + solve throughput (n=200,064 synthetic power grid)"
UNIT = "refactor+solve/s"
FP64_PEAK_TFLOPS = 1.254  # GB300 FP64 FMA rate measured by a standalone throughput probe (nominal 1.25)
L2_BYTES = 129 * 2**20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32+refinement and batched lines")
    ap.add_argument("--serve", action="store_true",
                    help="instead of the refactor+solve step: the continuous-batching serving loop on mixed "
                         "patterns with Poisson arrivals; prints p50/p99 latency")
    ap.add_argument("--serve-patterns", default="serve5k,serve20k,serve50k,serve100k,serve200k,serve500k")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="offered requests per second")
    ap.add_argument("--serve-requests", type=int, default=3000, help="timed requests (after a tenth as warm-up)")
    ap.add_argument("--serve-precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--batched", action="store_true",
                    help="instead of the step: the batched FP64 refactorization of 256 value sets of the "
                         "20k-unknown matrix, timed per factorization, with its bandwidth roofline")
    ap.add_argument("--sets", type=int, default=256, help="with --batched: the number of value sets")
    ap.add_argument("--latency", action="store_true",
                    help="instead of the step: the launch/latency-bound small patterns (32x32 grid in natural "
                         "order, the 5k serving pattern): microseconds per level against the floor of a CUDA "
                         "graph of as many dependent one-element kernels")
    ap.add_argument("--precision", metavar="WORKLOAD", default=None,
                    help="instead of the step: FP32 factor + FP64 refinement against FP64 and the CPU "
                         "oracle on one workload (backward errors, differences, times)")
    ap.add_argument("--factor-blocks", action="store_true",
                    help="with --precision or --analysis-only: the supernodal factorization (the "
                         "schedule that fits the 1000x1000 mesh with 256 nets)")
    ap.add_argument("--analysis-only", metavar="WORKLOAD", default=None,
                    help="instead of the step: the host analysis alone (host_only, no GPU), timed "
                         "--steps times after one untimed run")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        try:
            lines = open(self.out.name).read().strip().splitlines()
        except OSError:
            lines = []
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.out.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle
def cpu_oracle_steps(m, values, b, min_seconds=10.0, max_reps=5):
    """The oracle as it stands: single-threaded G/P factor + solves."""
    import oracle
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    reps, t0 = 0, time.perf_counter()
    while True:
        f.factor(values[reps % len(values)])
        f.solve(b)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    return reps / el, reps, el


def _oracle_refactor_worker(job):
    """One process of the parallel oracle baseline: the oracle's numeric
    refactorization of its share of the value sets, timed in the process."""
    name, seeds, sigma, base_seed = job
    import oracle
    m = synth.make(name, 1)
    vals = [m.values(s, sigma=sigma, base_seed=base_seed) for s in seeds]
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    t0 = time.perf_counter()
    for v in vals:
        f.factor(v)
    return time.perf_counter() - t0, len(vals)


def cpu_batched_baseline(name, seeds, sigma=0.1, base_seed=5, cores=None):
    """The oracle on a batch of same-pattern value sets, spread one process
    per host core (the sets are independent): sets / the slowest process's
    time.  Processes are spawned, never forked."""
    import multiprocessing as mp
    if cores is None:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = max(1, min(int(cores), len(seeds)))
    jobs = [(name, seeds[i::cores], sigma, base_seed) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_refactor_worker, jobs)
    slowest = max(t for t, _ in res)
    done = sum(c for _, c in res)
    return {"value": done / slowest if slowest > 0 else None, "unit": "refactorizations/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{done} value sets of {name} (the oracle's numeric refactorization), "
                      f"one process per core, {slowest:.2f} s for the slowest"}


def kernel_source_hash():
    """Hash of the file holding the level kernel (k_level)."""
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_1908_00204_gb300", "csrc", "kernels_factor.cu"), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(workload):
    """(DRAM bytes per refactorization's level sweep, note on the schedule it
    was captured with) from the committed ncu summary, if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"k_level_fp64_{workload}.traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_factor"), d.get("schedule")


# ------------------------------------------------------------------- arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    m = synth.make(args.workload, 1)
    values = [m.values(s) for s in VALUE_SEEDS]
    b = synth.rhs(m.n, args.nrhs, 7)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    for w in range(args.warmup):
        f.factor(values[w % len(values)])
        f.solve(b)
    t0 = time.perf_counter()
    for k in range(args.steps):
        f.factor(values[k % len(values)])
        f.solve(b)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n": m.n, "nrhs": args.nrhs},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full refactor+solve steps of the workload, single thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def extras(g, torch, dev, m, vals_host, b_host, h):
    """FP32 + FP64 refinement on the bench matrix, and batched refactorization
    of 256 Monte-Carlo value sets of the 20k-unknown matrix (FP64 and FP32 +
    refinement, 4 right-hand sides each) against one-at-a-time FP64."""
    out = {}

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ts))

    v = torch.from_numpy(vals_host[0]).to(dev)
    b = torch.from_numpy(b_host).to(dev)
    x = torch.empty_like(b)
    info = {}

    def ir():
        _, i = g.glu_solve_refine(h, b, x, tol=1e-12, maxit=20)
        info.update(i)
    g.glu_factor_f32(h, v)
    ir()
    f32 = timed(lambda: g.glu_factor_f32(h, v))
    s32 = timed(ir)
    out["fp32_refine"] = {"workload": m.stats()["rows"] and WORKLOAD, "factor_ms": f32,
                          "refine_solve_ms": s32, "refactor_solve_per_s": 1e3 / (f32 + s32),
                          "iterations": info.get("iterations"), "berr": info.get("berr")}
    mb = synth.make("mesh100x200_nets64", 1)
    B, K = 256, 4
    V = torch.from_numpy(np.stack([mb.values(100 + i, sigma=0.1, base_seed=5) for i in range(B)])).to(dev)
    R = torch.from_numpy(np.stack([synth.rhs(mb.n, K, 300 + i) for i in range(B)])).to(dev)
    hb = g.glu_analyze(mb.n, mb.colptr, mb.rowidx, mb.perm)
    g.glu_set_stream(hb, torch.cuda.current_stream(dev))
    v0, r0 = V[0].contiguous(), R[0].contiguous()
    g.glu_factor(hb, v0)
    g.glu_solve(hb, r0)
    single = timed(lambda: (g.glu_factor(hb, v0), g.glu_solve(hb, r0)))
    g.glu_factor_batched(hb, V)
    g.glu_solve_batched(hb, R)
    b64 = timed(lambda: (g.glu_factor_batched(hb, V), g.glu_solve_batched(hb, R)))
    binfo = {}

    def bir():
        g.glu_factor_batched_f32(hb, V)
        _, i = g.glu_solve_batched_refine(hb, R, tol=1e-12, maxit=20)
        binfo.update(i)
    bir()
    b32 = timed(bir)
    out["batched"] = {"workload": "mesh100x200_nets64", "n": mb.n, "sets": B, "nrhs": K,
                      "one_at_a_time_fp64_per_s": 1e3 / single, "fp64_batched_per_s": B * 1e3 / b64,
                      "fp32_refine_batched_per_s": B * 1e3 / b32, "fp64_batched_ms": b64, "fp32_refine_batched_ms": b32,
                      "refine_iterations": binfo.get("iterations"), "refine_berr": binfo.get("berr"),
                      "graph_launches_per_batched_factor": 1}
    g.glu_destroy(hb)
    out["serve"] = serve_compare(g, torch)
    return out


def serve_compare(g, torch, names=("serve5k", "serve20k", "serve50k"), nreq=800, load=0.7, seed=2027):
    """Continuous-batching serving against a plain loop that factors and
    solves one request at a time (FP64, one handle per pattern), on the same
    Poisson arrivals over mixed patterns with 1-8 right-hand sides.  The
    offered rate is `load` times the plain loop's measured capacity, so both
    arms keep up; latency is scheduled arrival -> result on the host, the
    first tenth of the requests excluded."""
    import collections
    from paper_1908_00204_gb300.serve import Request, Server
    dev = torch.device("cuda", torch.cuda.current_device())
    mats = {k: synth.make(k, 1) for k in names}
    pool = 8
    vals = {k: [m.values(100 + i, sigma=0.1, base_seed=7) for i in range(pool)] for k, m in mats.items()}
    rhs = {k: synth.rhs(m.n, 8, 11) for k, m in mats.items()}
    rng = np.random.default_rng(seed)
    nwarm = nreq // 10
    total = nreq + nwarm
    keys = [names[i] for i in rng.integers(len(names), size=total)]
    nrhs = rng.integers(1, 9, size=total)

    def make(i):
        k = keys[i]
        return Request(i, k, vals[k][i % pool], rhs[k][: int(nrhs[i])])
    # the plain arm's handles, and its service time per pattern
    handles = {}
    for k, m in mats.items():
        handles[k] = g.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
        g.glu_set_stream(handles[k], torch.cuda.current_stream(dev))

    def plain_one(req):
        h = handles[req.key]
        v = torch.from_numpy(req.values).to(dev, non_blocking=True)
        b = torch.from_numpy(np.ascontiguousarray(req.b)).to(dev, non_blocking=True)
        g.glu_factor(h, v)
        return g.glu_solve(h, b).cpu().numpy()
    svc = []
    for i in range(60):
        r = make(i)
        t = time.perf_counter()
        plain_one(r)
        svc.append(time.perf_counter() - t)
    capacity = 1.0 / float(np.mean(svc[10:]))
    rate = load * capacity
    arrivals = list(np.cumsum(rng.exponential(1.0 / rate, total)))
    # serving arm
    srv = Server(device_budget_bytes=60e9, max_batch=32, slots=4, replicas=3, batch_min=8)
    for k, m in mats.items():
        srv.register(k, m.n, m.colptr, m.rowidx, m.perm)
        srv.prepare(k, vals[k][0], rhs[k][:1])    # analyses, replicas and captured graphs before traffic
    batches0 = len(srv.batch_sizes)
    t0 = time.perf_counter()
    srv.run(arrivals, make)
    wall_s = time.perf_counter() - t0
    lat_s = srv.latencies(skip=nwarm) * 1e3
    ok_s = all(r.status == 0 for r in srv.done)
    # plain arm: the same arrivals, served in order, one at a time
    q = collections.deque()
    lat_p = np.empty(total)
    t0 = time.perf_counter()
    i = 0
    while i < total or q:
        now = time.perf_counter() - t0
        while i < total and arrivals[i] <= now:
            q.append(i)
            i += 1
        if not q:
            time.sleep(max(0.0, min(arrivals[i] - now, 0.001)))
            continue
        j = q.popleft()
        plain_one(make(j))
        lat_p[j] = time.perf_counter() - t0 - arrivals[j]
    wall_p = time.perf_counter() - t0
    lat_p = lat_p[nwarm:] * 1e3
    for h in handles.values():
        g.glu_destroy(h)

    def summary(lat, wall, extra):
        d = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
             "mean_ms": float(lat.mean()), "achieved_per_s": total / wall}
        d.update(extra)
        return d
    return {"patterns": {k: m.n for k, m in mats.items()}, "requests": nreq, "warmup_requests": nwarm,
            "nrhs": "uniform 1..8", "plain_capacity_per_s": capacity, "offered_per_s": rate, "load": load,
            "serving": summary(lat_s, wall_s, {"launches": len(srv.batch_sizes) - batches0, "all_ok": ok_s,
                                               "streams": 4, "max_batch": 32, "batch_min": 8, "replicas": 3,
                                               "batched_launches": int(sum(b > 1 for b in
                                                                           srv.batch_sizes[batches0:]))}),
            "plain_one_at_a_time_fp64": summary(lat_p, wall_p, {})}


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def roofline(achieved_tflops, traffic, fac_ms):
    """The level sweep against the FP64 pipe; its measured DRAM traffic (if
    the committed capture matches the kernel) also as a bandwidth fraction.
    ``traffic``: bytes per refactorization, or (bytes, note on the schedule
    the capture was taken with), or None."""
    note = None
    if isinstance(traffic, tuple):
        traffic, note = traffic
    r = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
         "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": traffic,
         "kernel": "k_level (FP64 level sweep of one refactorization)",
         "peak_source": "measured FP64 FMA throughput of a GB300 (standalone probe, "
                        "profiles/fp64_fma_peak_probe.md; MEASURED_PEAKS.json covers HBM and bf16 only)"}
    if note:
        r["traffic_schedule"] = note
    hbm = measured_hbm_gbs()
    if traffic is not None and fac_ms > 0:
        r["dram_gbs"] = traffic / (fac_ms * 1e-3) / 1e9
        if hbm:
            r["dram_frac_of_measured_hbm"] = r["dram_gbs"] / hbm
    return r


def max_over_ranks(ms, dist, device):
    """The slowest rank's time, on every rank (ms itself without a process group)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps, world, max_ms):
    """Whole-job throughput: each of the `world` replicas ran `steps` steps
    (weak scaling), the job took as long as the slowest rank."""
    return world * steps / (max_ms / 1e3)


def run_ours(args):
    import torch
    import paper_1908_00204_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.build.build()
    g.load_library()
    dev = torch.device("cuda", local)

    m = synth.make(args.workload, 1)
    vals_host = [m.values(s) for s in VALUE_SEEDS]
    b_host = synth.rhs(m.n, args.nrhs, 7)
    t0 = time.perf_counter()
    h = g.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    analyze_s = time.perf_counter() - t0
    st = g.glu_get_stats(h)
    stream = torch.cuda.current_stream(dev)
    g.glu_set_stream(h, stream)
    vals = [torch.from_numpy(v).to(dev) for v in vals_host]
    b = torch.from_numpy(b_host).to(dev)
    x = torch.empty_like(b)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    for w in range(max(args.warmup, 3)):
        g.glu_factor(h, vals[w % len(vals)])
        g.glu_solve(h, b, x)
    g.glu_sync(h)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = g.glu_get_stats(h)["kernel_launches"]
    with ClockSampler(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()                      # L2 flushed between steps (outside the events)
            e0, e1, e2 = ev[k]
            e0.record(stream)
            g.glu_factor(h, vals[k % len(vals)])
            e1.record(stream)
            g.glu_solve(h, b, x)
            e2.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if dist is not None:
            dist.barrier()
    g.glu_sync(h)
    launches = g.glu_get_stats(h)["kernel_launches"] - launches0
    clocks = clk.summary()
    fac = [e0.elapsed_time(e1) for e0, e1, _ in ev]
    sol = [e1.elapsed_time(e2) for _, e1, e2 in ev]
    total_ms = max_over_ranks(float(sum(f + s for f, s in zip(fac, sol))), dist, dev)
    value = job_rate(args.steps, world, total_ms)
    fac_ms = float(np.mean(fac))
    flops = st["flops"]
    achieved = flops / (fac_ms * 1e-3) / 1e12

    e2e = None
    if not args.no_e2e:
        vp = [torch.from_numpy(v).pin_memory() for v in vals_host]
        bp = torch.from_numpy(b_host).pin_memory()
        xp = torch.empty_like(bp).pin_memory()
        g.glu_factor(h, vp[0].numpy())
        g.glu_solve(h, bp.numpy(), xp.numpy())
        t0 = time.perf_counter()
        for k in range(args.steps):
            g.glu_factor(h, vp[k % len(vp)].numpy())      # H2D of the values inside
            g.glu_solve(h, bp.numpy(), xp.numpy())        # H2D of b, D2H of x inside
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(m.nnz * 8 + b_host.size * 8),
               "d2h_bytes_per_step": int(b_host.size * 8 + 2 * 8)}

    extra = None
    if rank == 0 and world == 1 and not args.no_extras:
        extra = extras(g, torch, dev, m, vals_host, b_host, h)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, reps, el = cpu_oracle_steps(m, vals_host, b_host)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{reps} full refactor+solve steps of the same workload ({el:.1f} s), single thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": m.n, "nnz_a": m.nnz, "nnz_lu": st["nnz_lu"],
                       "levels": st["nlevels"], "flops_per_factor": flops, "nrhs": args.nrhs,
                       "value_sets": len(VALUE_SEEDS), "l2": "flushed between steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "refactor_ms": fac_ms, "solve_ms": float(np.mean(sol)),
            "gflops_refactor": flops / (fac_ms * 1e-3) / 1e9,
            "analyze_s": analyze_s, "wall_s_timed_loop": wall,
            "roofline": roofline(achieved, traffic_for(args.workload), fac_ms),
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "extras": extra,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Requests (pattern uniform over the list, new values, 1-8 right-hand
    sides) arrive as a Poisson process at the offered rate; the serving loop
    batches same-pattern requests and overlaps patterns on streams.  Latency
    is submit -> result on the host, the first tenth of the requests being
    warm-up."""
    import torch
    import paper_1908_00204_gb300 as g
    from paper_1908_00204_gb300.serve import Request, Server
    names = args.serve_patterns.split(",")
    mats = {k: synth.make(k, 1) for k in names}
    pool = 16   # value sets per pattern, drawn in turn (consecutive requests of a pattern differ)
    vals = {k: [m.values(100 + i, sigma=0.1, base_seed=7) for i in range(pool)] for k, m in mats.items()}
    nwarm = max(args.serve_requests // 10, 1)
    nreq = args.serve_requests + nwarm
    rng = np.random.default_rng(2026)
    keys = [names[i] for i in rng.integers(len(names), size=nreq)]
    nrhs = rng.integers(1, 9, size=nreq)
    rhs = {k: synth.rhs(m.n, 8, 11) for k, m in mats.items()}

    def make(i):
        k = keys[i]
        return Request(i, k, vals[k][i % pool], rhs[k][: int(nrhs[i])])
    srv = Server(device_budget_bytes=60e9, max_batch=64, slots=4, precision=args.serve_precision, replicas=3,
                 batch_min=8)
    t0 = time.perf_counter()
    for k, m in mats.items():
        srv.register(k, m.n, m.colptr, m.rowidx, m.perm)
        srv.prepare(k, vals[k][0], rhs[k][:1])    # analyses, replicas and captured graphs before traffic
    setup_s = time.perf_counter() - t0
    arrivals = list(np.cumsum(rng.exponential(1.0 / args.serve_rate, nreq)))
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        srv.run(arrivals, make)
        wall = time.perf_counter() - t0
    clock = clk.summary()
    lat = srv.latencies(skip=nwarm) * 1e3
    line = {"metric": "serving latency, submit to result (mixed patterns, Poisson arrivals)",
            "value": float(np.percentile(lat, 99)), "unit": "ms (p99)", "higher_is_better": False,
            "p50_ms": float(np.percentile(lat, 50)), "p90_ms": float(np.percentile(lat, 90)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "offered_rate_per_s": args.serve_rate, "achieved_rate_per_s": nreq / wall,
            "requests": args.serve_requests, "warmup_requests": nwarm, "precision": args.serve_precision,
            "patterns": {k: {"n": m.n, "nnz_a": m.nnz} for k, m in mats.items()},
            "batches": srv.batches, "analyses": srv.analyses, "evictions": srv.evictions,
            "setup_s": setup_s, "wall_s": wall, "n_gpus": 1, "data": "synthetic", "clocks": clock,
            "config": {"workload": "serving " + ",".join(names), "nrhs": "uniform 1..8",
                       "values": f"{pool} Monte-Carlo value sets per pattern, drawn in turn",
                       "device_budget_gb": 60, "max_batch": 64, "streams": 4}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """The batched refactorization: 256 (--sets) Monte-Carlo value sets of the
    20k-unknown matrix in one graph launch, CUDA events per factorization, L2
    flushed between them.  Lanes run over value sets, so every update streams
    the target (read + write) and L(i,j) of 32 sets at a time: the algorithmic
    bytes per update and set are 16 (targets only, L from cache) to 24.  Also
    the batched solve of 4 right-hand sides per set, timed the same way."""
    B = max(1, args.sets)
    # the oracle baseline first: its processes start before any GPU call
    cpu = None if args.no_cpu_baseline else cpu_batched_baseline("mesh100x200_nets64",
                                                                 [100 + i for i in range(B)])
    import torch
    import paper_1908_00204_gb300 as g
    g.build.build()
    g.load_library()
    dev = torch.device("cuda", 0)
    mb = synth.make("mesh100x200_nets64", 1)
    V = torch.from_numpy(np.stack([mb.values(100 + i, sigma=0.1, base_seed=5) for i in range(B)])).to(dev)
    hb = g.glu_analyze(mb.n, mb.colptr, mb.rowidx, mb.perm)
    stream = torch.cuda.current_stream(dev)
    g.glu_set_stream(hb, stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        g.glu_factor_batched(hb, V)
    g.glu_sync(hb)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.glu_factor_batched(hb, V)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    g.glu_sync(hb)
    R = torch.from_numpy(np.stack([synth.rhs(mb.n, 4, 300 + i) for i in range(B)])).to(dev)
    g.glu_solve_batched(hb, R)
    torch.cuda.synchronize()
    ts_solve = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.glu_solve_batched(hb, R)
        e1.record(stream)
        torch.cuda.synchronize()
        ts_solve.append(e0.elapsed_time(e1))
    st = g.glu_get_stats(hb)
    ms = float(np.median(ts))
    upd = float(st["n_updates"]) * B
    hbm = measured_hbm_gbs()
    lo, hi = 16.0 * upd / (ms * 1e-3) / 1e9, 24.0 * upd / (ms * 1e-3) / 1e9
    line = {"metric": f"batched FP64 refactorizations per second ({B} value sets, n=20,064)",
            "value": B * 1e3 / ms, "unit": "refactorizations/s", "higher_is_better": True,
            "ms_per_batch": ms, "solve_ms_per_batch_4rhs": float(np.median(ts_solve)),
            "gflops": st["flops"] * B / (ms * 1e-3) / 1e9, "dtype": "f64",
            "roofline": {"bound": "hbm", "achieved": lo, "achieved_upper": hi, "peak": hbm, "unit": "GB/s",
                         "frac": lo / hbm if hbm else None, "frac_upper": hi / hbm if hbm else None,
                         "traffic": None, "kernel": "k_level_b (one level of the batched sweep)",
                         "algorithmic_bytes": "16-24 per update and value set (target read+write, L(i,j))",
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "config": {"workload": "mesh100x200_nets64", "sets": B, "updates_per_set": st["n_updates"],
                       "l2": "flushed between factorizations"},
            "cpu_baseline": cpu, "steps": args.steps, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    g.glu_destroy(hb)
    return 0


def run_latency(args):
    """Small patterns whose refactorization is a chain of short levels: the
    32 x 32 grid in natural order (1,024 levels of one column) and the
    5k-unknown serving pattern.  Per pattern: device time of one
    refactorization (one graph launch; the matrix stays in L2) and of one
    solve, the kernels one refactorization launches, and the floor -- a CUDA
    graph of as many dependent one-element kernels, timed the same way."""
    import torch
    import paper_1908_00204_gb300 as g
    g.build.build()
    g.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    reps = max(args.steps, 20)
    cases = []

    def median_ms(fn):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))
    for name in ("grid32_natural", "serve5k"):
        m = synth.make(name, 1)
        h = g.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
        g.glu_set_stream(h, stream)
        v = torch.from_numpy(m.values(7)).to(dev)
        b = torch.from_numpy(synth.rhs(m.n, 1, 7)).to(dev)
        x = torch.empty_like(b)
        for _ in range(max(args.warmup, 3)):
            g.glu_factor(h, v)
            g.glu_solve(h, b, x)
        g.glu_sync(h)
        torch.cuda.synchronize()
        k0 = g.glu_get_stats(h)["kernel_launches"]
        g.glu_factor(h, v)
        g.glu_sync(h)
        nk = int(g.glu_get_stats(h)["kernel_launches"] - k0)
        f_ms = median_ms(lambda: g.glu_factor(h, v))
        s_ms = median_ms(lambda: g.glu_solve(h, b, x))
        g.glu_sync(h)
        st = g.glu_get_stats(h)
        # the floor: nk dependent one-element kernels in one graph
        z = torch.zeros(1, device=dev)
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                z.add_(1.0)
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(nk):
                z.add_(1.0)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        floor_ms = median_ms(graph.replay)
        cases.append({"workload": name, "n": m.n, "levels": st["nlevels"],
                      "dense_block_columns": st["factor_tail_cols"], "kernels_per_refactor": nk,
                      "refactor_us": f_ms * 1e3, "us_per_kernel": f_ms * 1e3 / max(nk, 1),
                      "solve_us": s_ms * 1e3, "floor_us_per_node": floor_ms * 1e3 / max(nk, 1),
                      "refactor_over_floor": f_ms / floor_ms if floor_ms > 0 else None})
        g.glu_destroy(h)
        del graph
    line = {"metric": "latency-bound refactorization: microseconds per level kernel vs a graph-node floor",
            "unit": "us", "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"l2": "warm (the matrices fit in L2)", "reps": reps,
                       "floor": "CUDA graph of as many dependent one-element torch kernels"},
            "cases": cases}
    print(json.dumps(line), flush=True)
    return 0


def run_analysis_only(args):
    """The analysis of one workload on the host cores (option host_only: the
    fill, Algorithm 4, the levels and the schedules; nothing on the GPU),
    wall time per call."""
    import paper_1908_00204_gb300 as g
    g.build.build()
    m = synth.make(args.analysis_only, 1)
    opts = dict(host_only=1, factor_blocks=int(args.factor_blocks))
    times = []
    for k in range(max(args.steps, 1) + 1):
        t0 = time.perf_counter()
        h = g.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, g.default_options(**opts))
        dt = time.perf_counter() - t0
        st = g.glu_get_stats(h)
        g.glu_destroy(h)
        if k > 0:
            times.append(dt)
    out = {"metric": "host analysis time", "workload": args.analysis_only, "n": m.n, "nnz_a": m.nnz,
           "factor_blocks": int(args.factor_blocks), "threads": os.cpu_count(),
           "analyze_s_median": float(np.median(times)), "analyze_s": [round(t, 4) for t in times],
           "nnz_lu": st["nnz_lu"], "nlevels": st["nlevels"], "n_pairs": st["n_pairs"]}
    print(json.dumps(out), flush=True)


def run_precision(args):
    """FP32 factorization + FP64 iterative refinement to 1e-12 against the
    FP64 factorization and the CPU oracle on one workload: backward errors
    (host FP64), max differences of the solutions, times."""
    import scipy.sparse as sp
    import torch
    import oracle
    import paper_1908_00204_gb300 as g
    name = args.precision
    m = synth.make(name, 1)
    out = {"metric": "FP32 factor + FP64 refinement vs FP64 and the oracle", "workload": name,
           "n": m.n, "nnz_a": m.nnz, "factor_blocks": int(args.factor_blocks)}
    t0 = time.perf_counter()
    h = g.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, g.default_options(factor_blocks=int(args.factor_blocks)))
    out["analyze_s"] = time.perf_counter() - t0
    st = g.glu_get_stats(h)
    out.update({k: st[k] for k in ("nnz_lu", "nlevels", "n_updates", "flops", "device_bytes")})
    print(json.dumps({"analysis": out}), flush=True)
    v = m.values(4001)
    b = synth.rhs(m.n, 1, 4001)
    A = sp.csc_matrix((v, m.rowidx, m.colptr), shape=(m.n, m.n))
    anorm = abs(A).sum(axis=1).max()

    def berr(x):
        x = np.asarray(x).reshape(-1)
        bb = b.reshape(-1)
        return float(np.abs(bb - A @ x).max() / (anorm * np.abs(x).max() + np.abs(bb).max()))
    vd, bd = torch.from_numpy(v).cuda(), torch.from_numpy(b).cuda()
    for _ in range(2):
        g.glu_factor(h, vd)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    g.glu_factor(h, vd)
    e1.record()
    x64 = g.glu_solve(h, bd)
    e2.record()
    torch.cuda.synchronize()
    out["fp64_factor_ms"], out["fp64_solve_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
    x64h = x64.cpu().numpy().reshape(-1)
    out["fp64_berr"] = berr(x64h)
    g.glu_factor_f32(h, vd)
    torch.cuda.synchronize()
    e0.record()
    g.glu_factor_f32(h, vd)
    e1.record()
    x32, info = g.glu_solve_refine(h, bd, tol=1e-12, maxit=30)
    e2.record()
    torch.cuda.synchronize()
    out["fp32_factor_ms"], out["fp32_refine_solve_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
    out["refine"] = info
    x32h = x32.cpu().numpy().reshape(-1)
    out["fp32_refine_berr"] = berr(x32h)
    out["max_rel_diff_refined_vs_fp64"] = float(np.abs(x32h - x64h).max() / np.abs(x64h).max())
    t0 = time.perf_counter()
    xo = np.asarray(oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v).solve(b)).reshape(-1)
    out["oracle_s"] = time.perf_counter() - t0
    out["oracle_berr"] = berr(xo)
    out["max_rel_diff_fp64_vs_oracle"] = float(np.abs(x64h - xo).max() / np.abs(xo).max())
    out["max_rel_diff_refined_vs_oracle"] = float(np.abs(x32h - xo).max() / np.abs(xo).max())
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.analysis_only:
        return run_analysis_only(args)
    if args.precision:
        return run_precision(args)
    if args.batched:
        return run_batched(args)
    if args.latency:
        return run_latency(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
