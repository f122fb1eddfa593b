#!/usr/bin/env python3
"""Benchmark: all 73 per-vertex orbit counts of one synthetic graph per step.

Default workload: Chung-Lu graph, n = 1,000,000, ~10,000,000 edges, degree
exponent 2.1, degrees capped at 5,000 (seeded), uint32 CSR resident in HBM.
One step = one evoke_count_orbits call (every pass of the path, DAG build to
the int64[n x 73] induced counts).  Metric: edges per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl evoke|reference]

N > 1 runs under torch.distributed (one rank per GPU, replicas of the same
workload on independent seeds: weak scaling, no data-path collective).
``--impl reference`` times the CPU oracle (tests' reference implementation)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
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

METRIC = "edges/s to all 73 vertex orbits"
UNIT = "edges/s"

WORKLOADS = {
    # name: (generator kwargs, description)
    "chung_lu_1m": (dict(kind="chung_lu", n=1_000_000, m=10_000_000, exponent=2.1, cap=5000),
                    "Chung-Lu n=1,000,000 m~10,000,000 exponent 2.1 degree cap 5,000"),
    "er_2000": (dict(kind="er", n=2000, m=10000),
                "Erdos-Renyi G(n=2000, m=10000)"),
    "chung_lu_100k": (dict(kind="chung_lu", n=100_000, m=1_000_000, exponent=2.1, cap=5000),
                      "Chung-Lu n=100,000 m~1,000,000 exponent 2.1 degree cap 5,000"),
    "chung_lu_30k": (dict(kind="chung_lu", n=30_000, m=300_000, exponent=2.1, cap=1000),
                     "Chung-Lu n=30,000 m~300,000 exponent 2.1 degree cap 1,000"),
    "batch_200k": (dict(kind="batch", graphs=200_000, nmin=10, nmax=500),
                   "200,000 graphs, n ~ U[10,500], 1/3 each ER (avg degree 4-12), BA (m0 2-5), "
                   "2-D RGG (avg degree 6); one CUDA-graph replay per step"),
    "rmat_20": (dict(kind="rmat", scale=20, edge_factor=16, cap=20000),
                "R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), degree cap 20,000"),
    "rmat_20_learned": (dict(kind="learned", scale=20, edge_factor=16, cap=20000, train=20,
                             train_scales=(16, 17, 18)),
                        "R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
                        "degree cap 20,000; learned vs degree-bucket schedule (MLP 4-32-32-1 "
                        "trained on 20 R-MAT scale 16-18 graphs)"),
    "rmat_16_learned": (dict(kind="learned", scale=16, edge_factor=16, cap=20000, train=4,
                             train_scales=(13, 14)),
                        "R-MAT scale 16 (small learned-schedule check)"),
    "batch_20k": (dict(kind="batch", graphs=20_000, nmin=10, nmax=500),
                  "20,000 graphs, n ~ U[10,500], 1/3 each ER / BA / RGG"),
    "chung_lu_1m_four": (dict(kind="chung_lu", n=1_000_000, m=10_000_000, exponent=2.1,
                              cap=5000, orbits=15),
                         "Chung-Lu n=1,000,000 m~10,000,000 exponent 2.1 degree cap 5,000; "
                         "4-vertex orbits 0-14 only"),
}
METRIC_FOUR = "edges/s to the 15 vertex orbits of 2- to 4-vertex graphlets"


METRIC_BATCH = "batched graphs/s, all 73 vertex orbits"


def metric_of(spec):
    if spec["kind"] == "batch":
        return METRIC_BATCH
    if spec["kind"] == "learned":
        return METRIC + " (learned schedule)"
    return METRIC_FOUR if spec.get("orbits", 73) == 15 else METRIC


def unit_of(spec):
    return "graphs/s" if spec["kind"] == "batch" else UNIT


def make_graph(spec, seed):
    from paper_1911_10616_gb300 import graphgen as gg
    if spec["kind"] == "rmat":
        return gg.rmat(spec["scale"], spec["edge_factor"], 0.57, 0.19, 0.19, seed, cap=spec["cap"])
    if spec["kind"] == "chung_lu":
        return gg.chung_lu(spec["n"], spec["m"], spec["exponent"], spec["cap"], seed)
    if spec["kind"] == "er":
        return gg.er_gnm(spec["n"], spec["m"], seed)
    raise ValueError(spec)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def root_pass_entries(g, T_slot):
    """Adjacency entries the per-root pass must stream for this graph: the
    wedge lists twice (sum over u of sum_{v in N(u)} d(v), i.e. sum d^2), the
    triangle lists of the edges opposite each vertex in its triangles
    (sum_e T(e)^2) and the out-lists of the directed 3-path enumeration (DP)."""
    d = g.degrees().astype(np.int64)
    sumd2 = int((d * d).sum())
    tri2 = int((T_slot.astype(np.int64) ** 2).sum() // 2)
    e = g.edges()
    a, b = e[:, 0], e[:, 1]
    fwd = (d[a] < d[b]) | ((d[a] == d[b]) & (a < b))
    src = np.where(fwd, a, b)
    dst = np.where(fwd, b, a)
    dplus = np.bincount(src, minlength=g.n).astype(np.int64)
    sk = np.bincount(src, weights=dplus[dst].astype(np.float64), minlength=g.n)
    dp = int((dplus.astype(np.float64) * sk).sum())
    return {"sum_d2": sumd2, "sum_T2": tri2, "DP": dp, "entries": 2 * sumd2 + tri2 + dp}


def cpu_oracle_baseline(spec_name, seed, budget_s=20.0):
    """Time the oracle as it stands on a bounded sample of the workload: the
    same generator at a reduced vertex/edge count, grown until the run takes
    a few seconds (bounded by budget_s)."""
    import oracle
    from paper_1911_10616_gb300 import graphgen as gg
    spec = dict(WORKLOADS[spec_name][0])
    threads = oracle.max_threads()
    method = oracle.formulas4 if spec.get("orbits", 73) == 15 else oracle.formulas
    if spec["kind"] == "batch":
        # graphs of the same generator, one by one, until the budget is used
        graphs = gg.small_graph_batch(400, spec["nmin"], spec["nmax"], seed)
        t0 = time.perf_counter()
        done = 0
        for gr in graphs:
            method(gr, threads)
            done += 1
            if time.perf_counter() - t0 > budget_s / 2:
                break
        dt = time.perf_counter() - t0
        return {"value": done / dt, "unit": "graphs/s", "cores": threads, "kind": "oracle",
                "sample": f"{done} graphs of the same generator (n ~ U[{spec['nmin']},{spec['nmax']}])",
                "seconds": dt}
    if spec["kind"] == "learned":  # the R-MAT graph of the learned-schedule workload
        spec = {"kind": "rmat", "scale": spec["scale"], "edge_factor": spec["edge_factor"],
                "cap": spec["cap"]}
    if spec["kind"] == "rmat":
        for scale in range(10, spec["scale"] + 1):
            g = make_graph(dict(spec, scale=scale), seed)
            t0 = time.perf_counter()
            method(g, threads)
            dt = time.perf_counter() - t0
            best = {"value": g.m / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                    "sample": f"the same generator at scale {scale} ({g})", "seconds": dt}
            if dt * 4 > budget_s:
                break
        return best
    if spec["kind"] == "er":
        g = make_graph(spec, seed)
        t0 = time.perf_counter()
        method(g, threads)
        dt = time.perf_counter() - t0
        return {"value": g.m / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": f"the full workload ({g})", "seconds": dt}
    frac = 0.005
    best = None
    while True:
        sub = dict(spec)
        sub["n"] = max(1000, int(spec["n"] * frac))
        sub["m"] = max(5000, int(spec["m"] * frac))
        g = make_graph(sub, seed)
        t0 = time.perf_counter()
        method(g, threads)
        dt = time.perf_counter() - t0
        best = {"value": g.m / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": (f"same generator at {frac:.3g} of the vertices and edges "
                           f"({g}, degree cap {spec['cap']})"), "seconds": dt}
        if dt * 4 > budget_s or frac >= 0.1:
            return best
        frac *= 2


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, on rank 0 only."""
    if rank != 0:
        return
    spec_name = args.workload
    res = []
    cb = None
    for step in range(args.warmup + args.steps):
        cb = cpu_oracle_baseline(spec_name, seed=1, budget_s=args.cpu_budget)
        if step >= args.warmup:
            res.append(cb)
    secs = [r["seconds"] for r in res]
    value = statistics.median([r["value"] for r in res])
    line = {
        "impl": "reference", "metric": metric_of(WORKLOADS[spec_name][0]), "value": value,
        "unit": unit_of(WORKLOADS[spec_name][0]),
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.median(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOADS[spec_name][1], "sample": cb["sample"]},
        "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample")} | {"value": value,
                                                                          "unit": cb["unit"]},
        "e2e": {"value": value, "unit": cb["unit"], "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def local_device() -> int:
    return int(os.environ.get("LOCAL_RANK", "0"))


def timed(fn, steps, stream, barrier):
    """Run fn() `steps` times between CUDA events on `stream`; seconds."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    barrier()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    barrier()
    return a.elapsed_time(b) / 1000.0


def max_over_ranks(x, dist):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


PROFILE_DRAM = {
    # workload -> committed ncu summary holding the root kernel's DRAM bytes
    "chung_lu_1m": "profiles/root_kernel_dram_chung_lu_1m.md",
}


def measured_traffic(workload):
    """dram__bytes_read.sum + dram__bytes_write.sum of one root_kernel launch
    from the committed ncu summary, or None when there is none or the kernel
    source changed since it was captured (the summary records its sha1)."""
    import hashlib
    import re
    rel = PROFILE_DRAM.get(workload)
    if rel is None or not os.path.exists(os.path.join(ROOT, rel)):
        return None
    text = open(os.path.join(ROOT, rel)).read()
    t = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    h = re.search(r"k_root_cu_sha1:\s*([0-9a-f]{40})", text)
    if not t or not h:
        return None
    src = os.path.join(ROOT, "paper_1911_10616_gb300", "csrc", "k_root.cu")
    if hashlib.sha1(open(src, "rb").read()).hexdigest() != h.group(1):
        return None
    return int(t.group(1))


def roofline_of(phases, g, ev, rp, col, n, m, args, four=False):
    peak, peak_kind = read_peaks()
    if not phases:
        return None
    name, (nl, calls, ms) = max(phases.items(), key=lambda kv: kv[1][2])
    per_launch_s = ms / 1000.0 / max(nl, 1)
    ent = None
    if name == "root" and g is not None and not args.no_roofline:
        if four:  # one wedge sweep (W and C4(u)) and nothing else
            d = g.degrees().astype(np.int64)
            ent = {"sum_d2": int((d * d).sum())}
            ent["entries"] = ent["sum_d2"]
        else:
            T_slot = ev.edge_orbits(rp, col, n, m)["T"].cpu().numpy()
            ent = root_pass_entries(g, T_slot)
        alg_bytes = 4 * ent["entries"]
    else:
        alg_bytes = 4 * (2 * m) + 8 * n  # lower bound: one read of the CSR
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = measured_traffic(args.workload) if name == "root" else None
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
            "algorithmic_bytes": alg_bytes, "launch_ms": per_launch_s * 1000.0, "units": ent}


def run_single(args, rank, world, dist, barrier):
    import torch
    import paper_1911_10616_gb300 as ev
    from paper_1911_10616_gb300 import _lib

    spec, desc = WORKLOADS[args.workload]
    orbits = spec.get("orbits", 73)
    seed = 1 + rank
    t0 = time.perf_counter()
    g = make_graph(spec, seed)
    gen_s = time.perf_counter() - t0
    ev.load()
    rp, col = ev.to_device(g)
    n, m = g.n, g.m
    stream = torch.cuda.current_stream()
    plan = ev.Plan.single(rp, col, n, m, validate=True, orbits=orbits)
    out = plan.new_output()
    plan.execute(out)
    # autotune the per-root pass shape (threads per CTA x persistent CTAs),
    # unless --root-shape fixes it
    sms = torch.cuda.get_device_properties(local_device()).multi_processor_count
    info0 = plan.info()
    shapes = ((512, 2 * sms), (1024, sms), (256, 4 * sms))
    if args.root_shape:
        th, ct = (int(x) for x in args.root_shape.split("x"))
        shapes = ((th, ct),)
    tune = []
    for th, ct in shapes:
        if ct > info0["root_ctas_max"]:
            continue
        plan.set_tuning(th, ct)
        tune.append((timed(lambda: plan.execute(out), 1, stream, barrier) if len(shapes) > 1 else 0.0,
                     th, ct))
    best = min(tune)
    plan.set_tuning(best[1], best[2])
    # autotune the root order (degree buckets, or grouped by highest-degree
    # neighbour in chunks of 16), unless --schedule fixes it
    orders = {"degree": ((0, 1),), "hub": ((1, 16),)}.get(args.schedule, ((0, 1), (1, 16)))
    sched_t = []
    for sched, chunk in orders:
        plan.set_schedule(sched, chunk)
        sched_t.append((timed(lambda: plan.execute(out), 1, stream, barrier) if len(orders) > 1 else 0.0,
                        sched, chunk))
    best_sched = min(sched_t)
    plan.set_schedule(best_sched[1], best_sched[2])
    for _ in range(args.warmup):
        plan.execute(out)
    barrier()

    # timed region: K executions of the whole pass sequence, inputs resident,
    # per-phase CUDA events recorded on the launching stream
    _lib.profile_reset()
    _lib.profile_enable(True)
    launches0 = _lib.launch_count()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t_run = timed(lambda: plan.execute_profiled(out), args.steps, stream, barrier)
    _lib.profile_enable(False)
    launches = _lib.launch_count() - launches0
    phases = _lib.profile_read()
    t_max = max_over_ranks(t_run, dist)
    value = world * m * args.steps / t_max

    # the same executions replayed as one CUDA graph each
    plan.launch_graph(out)
    t_graph = max_over_ranks(timed(lambda: plan.launch_graph(out), args.steps, stream, barrier), dist)

    # end to end through the public one-shot API: pinned host CSR in, host counts out
    e2e = None
    if args.e2e_steps > 0:
        h_rp = torch.from_numpy(g.rowptr.astype(np.uint32).view(np.int32)).pin_memory()
        h_col = torch.from_numpy(g.col.astype(np.uint32).view(np.int32)).pin_memory()
        h_out = torch.empty((n, orbits), dtype=torch.int64).pin_memory()
        d_rp = torch.empty_like(rp)
        d_col = torch.empty_like(col)

        def e2e_step():
            d_rp.copy_(h_rp, non_blocking=True)
            d_col.copy_(h_col, non_blocking=True)
            ev.count_orbits(d_rp, d_col, n, m, out=out, orbits=orbits, schedule=best_sched[1])
            h_out.copy_(out, non_blocking=True)

        e2e_t = max(max_over_ranks(timed(e2e_step, args.e2e_steps, stream, barrier), dist), 1e-12)
        e2e = {"value": world * m * args.e2e_steps / e2e_t, "unit": UNIT,
               "h2d_bytes_per_step": h_rp.numel() * 4 + h_col.numel() * 4,
               "d2h_bytes_per_step": h_out.numel() * 8}
    if rank != 0:
        return None
    info = plan.info()
    roof = roofline_of(phases, g, ev, rp, col, n, m, args, four=orbits == 15)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_oracle_baseline(args.workload, seed=1, budget_s=args.cpu_budget)
            cpu.pop("seconds", None)
        except Exception as exc:  # report, never fake
            cpu = {"error": repr(exc)}
    return {
        "metric": metric_of(spec), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": desc, "n": n, "m": m, "seed": seed,
                   "parallelism": f"replicas{world}",
                   "schedule": ("degree-bucket" if best_sched[1] == 0 else
                                f"grouped by highest-degree neighbour, chunks of {best_sched[2]}"),
                   "schedule_s": {("degree-bucket" if sc == 0 else f"hub-grouped/{ch}"): round(t, 4)
                                  for t, sc, ch in sched_t},
                   "l2": "working set (CSR + per-edge arrays, GBs) far larger than the 129 MB L2",
                   "triangles": info["triangles"], "max_degree": info["max_degree"],
                   "tuned_root": {"threads": best[1], "ctas": best[2]},
                   "tuning_s": {f"{th}x{ct}": round(t, 4) for t, th, ct in tune},
                   "gen_s": round(gen_s, 1)},
        "graph_replay": {"value": world * m * args.steps / t_graph, "unit": UNIT,
                         "ms_per_step": 1000.0 * t_graph / args.steps},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "phases_ms": {k: round(v[2] / max(v[1], 1), 3) for k, v in sorted(phases.items())},
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }


def run_batch(args, rank, world, dist, barrier):
    import torch
    import paper_1911_10616_gb300 as ev
    from paper_1911_10616_gb300 import _lib, graphgen as gg

    spec, desc = WORKLOADS[args.workload]
    seed = 1 + rank
    t0 = time.perf_counter()
    rpc, colc, vo, eo = gg.small_graph_batch_tensors(spec["graphs"], spec["nmin"], spec["nmax"],
                                                     seed, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    G = vo.numel() - 1
    N = int(vo[-1].item())
    M = int(eo[-1].item()) // 2
    ev.load()
    stream = torch.cuda.current_stream()
    plan = ev.Plan.batch(rpc, colc, vo, eo, validate=True)
    out = plan.new_output()
    info = plan.info()

    # autotune the per-root pass: threads per CTA and persistent CTAs
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cands = [(512, 2 * sms), (256, 4 * sms), (128, 8 * sms), (64, 16 * sms), (64, 12 * sms)]
    tune = []
    for th, ct in cands:
        if ct > info["root_ctas_max"]:
            continue
        plan.set_tuning(th, ct)
        plan.execute(out)
        tune.append((timed(lambda: plan.execute(out), 1, stream, barrier), th, ct))
    best = min(tune)
    plan.set_tuning(best[1], best[2])

    for _ in range(args.warmup):
        plan.launch_graph(out)
    barrier()
    launches0 = _lib.launch_count()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t_run = timed(lambda: plan.launch_graph(out), args.steps, stream, barrier)
    launches = _lib.launch_count() - launches0
    t_max = max_over_ranks(t_run, dist)
    value = world * G * args.steps / t_max

    # per-phase times of one profiled execution (for the roofline)
    _lib.profile_reset()
    _lib.profile_enable(True)
    timed(lambda: plan.execute_profiled(out), 1, stream, barrier)
    _lib.profile_enable(False)
    phases = _lib.profile_read()

    # one launch sequence per graph, on a prefix of the batch
    k = min(args.per_graph_sample, G)
    h_vo, h_eo = vo.cpu().numpy(), eo.cpu().numpy()
    h_rp, h_col = rpc.cpu().numpy(), colc.cpu().numpy()
    singles = []
    for gi in range(k):
        gr = gg.batch_graph(h_rp, h_col, h_vo, h_eo, gi)
        singles.append((ev.to_device(gr), gr.n, gr.m))
    o1 = torch.empty((int(h_vo[k] - h_vo[0]) if k else 0, 73), dtype=torch.int64, device="cuda")

    def per_graph():
        for (drp, dcol), n1, m1 in singles:
            ev.count_orbits(drp, dcol, n1, m1, out=o1[: n1] if n1 else o1[:0])

    t_single = timed(per_graph, 1, stream, barrier) if k else None
    if rank != 0:
        return None
    roof = roofline_of(phases, None, ev, None, None, N, M, args)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        th = oracle.max_threads()
        kk = min(60, G)
        t0 = time.perf_counter()
        for gi in range(kk):
            oracle.formulas(gg.batch_graph(h_rp, h_col, h_vo, h_eo, gi), th)
        dt = time.perf_counter() - t0
        cpu = {"value": kk / dt, "unit": "graphs/s", "cores": th, "kind": "oracle",
               "sample": f"the first {kk} graphs of the batch"}
    return {
        "metric": "batched graphs/s, all 73 vertex orbits", "value": value, "unit": "graphs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": desc, "graphs": G, "vertices": N, "edges": M, "seed": seed,
                   "parallelism": f"replicas{world}", "max_component": info["max_component"],
                   "triangles": info["triangles"], "device_bytes": info["device_bytes"],
                   "tuned_root": {"threads": best[1], "ctas": best[2]},
                   "tuning_s": {f"{th}x{ct}": round(t, 4) for t, th, ct in tune},
                   "l2": "working set (tens of GB) far larger than the 129 MB L2",
                   "gen_s": round(gen_s, 1)},
        "edges_per_s": world * M * args.steps / t_max,
        "one_launch_per_graph": ({"graphs": k, "value": k / t_single, "unit": "graphs/s",
                                  "speedup_of_batched": (value / world) / (k / t_single)}
                                 if t_single else None),
        "e2e": None,
        "gpu_launches": launches,
        "roofline": roof,
        "phases_ms": {k2: round(v[2] / max(v[1], 1), 3) for k2, v in sorted(phases.items())},
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }


def run_learned(args, rank, world, dist, barrier):
    """Learned vs degree-bucket schedule on one R-MAT graph (same plan, same
    counts; only the persistent root queue's order differs)."""
    import torch
    import paper_1911_10616_gb300 as ev
    from paper_1911_10616_gb300 import _lib, graphgen as gg, learned

    spec, desc = WORKLOADS[args.workload]
    ev.load()
    t0 = time.perf_counter()
    train_graphs = learned.training_graphs(spec["train"], scales=spec["train_scales"],
                                           cap=spec["cap"], seed0=100 + 1000 * rank)
    data = [learned.measure(g)[:2] for g in train_graphs]
    collect_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, losses = learned.train(data, epochs=40, batch=4096)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    g = gg.rmat(spec["scale"], spec["edge_factor"], *learned.RMAT_ABC, seed=1 + rank,
                cap=spec["cap"])
    rp, col = ev.to_device(g)
    n, m = g.n, g.m
    stream = torch.cuda.current_stream()
    plan = ev.Plan.single(rp, col, n, m, validate=True)
    out = plan.new_output()
    res = {}
    for name, model in (("degree_bucket", None), ("learned", params)):
        plan.set_model(model)
        for _ in range(args.warmup):
            plan.execute(out)
        _lib.profile_reset()
        _lib.profile_enable(True)
        launches0 = _lib.launch_count()
        with ClockSampler(local_device()) as clk:
            t = timed(lambda: plan.execute_profiled(out), args.steps, stream, barrier)
        launches = _lib.launch_count() - launches0
        _lib.profile_enable(False)
        ph = _lib.profile_read()
        cyc, ends = plan.root_timing(out)
        e = ends.cpu().numpy().astype(np.float64)
        res[name] = {"ms_per_step": 1000.0 * t / args.steps,
                     "root_ms": ph["root"][2] / max(ph["root"][1], 1),
                     "tail_ms": float((e.max() - e.min()) / 1e6),
                     "cycles": cyc.cpu().numpy(), "phases": ph, "launches": launches,
                     "clocks": clk.summary()}
    X, y, _ = learned.measure(g)
    pred = _lib.mlp_forward(X, params).cpu().numpy()
    meas = y.cpu().numpy()
    busy = g.degrees() > 0
    work = learned.wedge_work(g)
    A = np.vstack([np.log2(1 + work[busy]), np.ones(busy.sum())]).T
    coef = np.linalg.lstsq(A, meas[busy], rcond=None)[0]
    ctas = plan.info()["root_ctas"]
    c = res["degree_bucket"]["cycles"].astype(np.float64)
    sim = {k: learned.list_schedule_makespan(c, o, ctas) / max(c.sum() / ctas, c.max())
           for k, o in (("learned", np.argsort(-pred, kind="stable")),
                        ("degree_bucket", np.argsort(-work, kind="stable")),
                        ("vertex_id", np.arange(n)))}
    plan.destroy()
    if rank != 0:
        return None
    roof = roofline_of(res["learned"]["phases"], g, ev, rp, col, n, m, args)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_oracle_baseline(args.workload, seed=1, budget_s=args.cpu_budget)
            cpu.pop("seconds", None)
        except Exception as exc:  # report, never fake
            cpu = {"error": repr(exc)}
    t_l = res["learned"]["ms_per_step"] / 1000.0
    return {
        "metric": metric_of(spec), "value": world * m / t_l, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["learned"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": desc, "n": n, "m": m, "max_degree": int(g.degrees().max()),
                   "training_vertices": int(sum(d[0].shape[0] for d in data)),
                   "collect_s": round(collect_s, 1), "train_s": round(train_s, 2),
                   "loss_first_last": [losses[0], losses[-1]]},
        "learned_vs_degree_bucket": {
            "step_speedup": res["degree_bucket"]["ms_per_step"] / res["learned"]["ms_per_step"],
            "root_pass_speedup": res["degree_bucket"]["root_ms"] / res["learned"]["root_ms"],
            "degree_bucket": {k: v for k, v in res["degree_bucket"].items()
                              if k in ("ms_per_step", "root_ms", "tail_ms")},
            "learned": {k: v for k, v in res["learned"].items()
                        if k in ("ms_per_step", "root_ms", "tail_ms")},
            "spearman_log2_cycles": {"learned": learned.spearman(pred[busy], meas[busy]),
                                     "wedge_work": learned.spearman(work[busy], meas[busy])},
            "mae_log2_cycles": {"learned": float(np.abs(pred[busy] - meas[busy]).mean()),
                                "wedge_work_affine": float(np.abs(A @ coef - meas[busy]).mean())},
            "simulated_makespan_over_lower_bound": sim},
        "e2e": None, "gpu_launches": res["learned"]["launches"], "roofline": roof,
        "phases_ms": {k2: round(v[2] / max(v[1], 1), 3)
                      for k2, v in sorted(res["learned"]["phases"].items())},
        "cpu_baseline": cpu, "clocks": res["learned"]["clocks"],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="evoke", choices=["evoke", "reference"])
    ap.add_argument("--workload", default="chung_lu_1m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--per-graph-sample", type=int, default=500)
    ap.add_argument("--root-shape", default="",
                    help="fix the per-root pass shape, THREADSxCTAS (default: autotune)")
    ap.add_argument("--schedule", default="auto", choices=["auto", "degree", "hub"],
                    help="fix the root order (default: autotune)")
    ap.add_argument("--no-roofline", action="store_true",
                    help="skip the extra pass that sizes the roofline's algorithmic bytes")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if WORKLOADS[args.workload][0]["kind"] == "batch":
        line = run_batch(args, rank, world, dist, barrier)
    elif WORKLOADS[args.workload][0]["kind"] == "learned":
        line = run_learned(args, rank, world, dist, barrier)
    else:
        line = run_single(args, rank, world, dist, barrier)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
