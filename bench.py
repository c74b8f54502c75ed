#!/usr/bin/env python
"""Benchmark of the GB300 ASCI search: scored excitations/s at (24e,30o).

One step is one full search (Algorithm 2 with Eq. 1, constraint batched) over
the synthetic Cr2-shaped workload: 30 orbitals, 12 alpha + 12 beta electrons,
|psi| = 1e6, C = 1e5 core determinants, N = 1e6 selected; C * n_exc =
6.73e9 scored excitations per step.  Inputs are device-resident when the timed
region starts; L2 is flushed (a 512 MB write) before every timed step, outside
the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl asci|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica (the search shards by constraint class with no data-path exchange);
timing is the max over ranks and `value` counts all ranks' excitations.
`--impl reference` times the plain CPU oracle on bounded samples of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ASCI search scored excitations/s at (24e,30o)"
# DRAM bytes (read + write) per staged pair reduced by the tile kernel k_cells,
# from one ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum over every tile launch of one search, divided by its
# staged pairs); `traffic` is this figure scaled to one launch, and null for
# a workload without a capture.
TILE_DRAM_BYTES_PER_RECORD = {"random_24e30o": 17.46}
TILE_DRAM_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum over the 42 launches of the "
                    "1024-record tile kernel in one search of the same workload at C = 1e4 with "
                    "2^25-pair batches (11.72 GB for 6.715e8 staged pairs)")
UNIT = "excitations/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="asci", choices=["asci", "reference"])
    p.add_argument("--workload", default="random_24e30o",
                   help="a single-system workload, or batched512 for 512 small systems")
    p.add_argument("--eps", type=float, default=0.0)
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32_fp64acc", "fp32_comp"])
    p.add_argument("--sharded", action="store_true",
                   help="under torchrun: one search split over the ranks by constraint class "
                        "(strong scaling) instead of one search per rank")
    p.add_argument("--pt2-workload", default="random_24e30o",
                   help="system of --workload pt2 (its psi and core size)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-rows", action="store_true",
                   help="skip the extra measured rows (eps 1e-10, FP32 variants, configs 1-2)")
    p.add_argument("--C", type=int, default=0,
                   help="core size override (0: the workload's); for profiling a smaller case")
    p.add_argument("--max-batch-pairs", type=int, default=0,
                   help="constraint-batch cap in pairs (0: sized from free memory)")
    p.add_argument("--cpu-sample-core", type=int, default=0,
                   help="core dets in each oracle sample (0: sized to ~10 s)")
    return p.parse_args()


# ----------------------------------------------------------------- clocks ---

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- workload ---

def load_workload(name):
    import numpy as np
    import workloads as W
    w = W.WORKLOADS[name]
    h1, eri, ec = w.integrals()
    A, B, c = w.psi()
    return w, h1, eri, ec, A, B, c, W.stored_e0(name), np


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# -------------------------------------------------------------- reference ---

def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_sample(w, h1, eri, ec, A, B, c, E0, core, np, threads=1):
    """Time the oracle (as it stands) on the top `core` core dets of the
    workload, single-core or its all-core form (`threads`)."""
    import oracle
    ints = oracle.Ints(h1, eri, ec)
    t0 = time.perf_counter()
    r = oracle.search(ints, A, B, c, E0, core, threads=threads)
    dt = time.perf_counter() - t0
    return r.generated, dt


def oracle_rows_per_s(h1, eri, ec, A, B, rows=16):
    """The oracle (as it stands) forming dense Hamiltonian rows of a
    determinant list: rows per second on one host core, over `rows` rows."""
    import numpy as np
    import oracle
    oracle.build()
    ints = oracle.Ints(h1, eri, ec)
    rows = min(rows, len(A))
    t0 = time.perf_counter()
    oracle.h_rows(ints, A, B, np.arange(rows))
    return rows / (time.perf_counter() - t0)


def oracle_pt2_rate(w, h1, eri, ec, A, B, c, E0, core):
    """The oracle's ASCI-PT2 on the top `core` core determinants: excitations
    per second on one host core."""
    import oracle
    import workloads as W
    oracle.build()
    t0 = time.perf_counter()
    oracle.pt2(oracle.Ints(h1, eri, ec), A, B, c, E0, core)
    return core * W.n_excitations(w.norb, w.na, w.nb) / (time.perf_counter() - t0)


def size_cpu_sample(w, args, threads=1):
    if args.cpu_sample_core:
        return args.cpu_sample_core
    # about 10-15 s of oracle work on this host class (measured ~7e5 pairs/s
    # per core; the all-core form scales to about half of the cores' sum)
    from math import ceil
    import workloads as W
    nexc = W.n_excitations(w.norb, w.na, w.nb)
    scale = 1.0 if threads <= 1 else max(1.0, 0.5 * threads)
    return max(1, min(w.C, int(ceil(1.0e7 * scale / nexc))))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, h1, eri, ec, A, B, c, E0, np = load_workload(args.workload)
    import oracle
    oracle.build()
    cores = host_cores()
    core = size_cpu_sample(w, args, cores)
    for _ in range(args.warmup):
        cpu_sample(w, h1, eri, ec, A, B, c, E0, max(1, core // 10), np, cores)
    tot_pairs, tot_t = 0, 0.0
    for _ in range(args.steps):
        p, dt = cpu_sample(w, h1, eri, ec, A, B, c, E0, core, np, cores)
        tot_pairs += p
        tot_t += dt
    value = tot_pairs / tot_t
    sample = (f"all-core oracle ({cores} threads) on the top {core} of {w.C} core dets of "
              f"{w.name} per step ({tot_pairs // args.steps} excitations/step), full psi for "
              f"exclusion")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "norb": w.norb, "nelec": [w.na, w.nb], "ndets": w.ndets,
                   "C": w.C, "N": w.N, "eps": args.eps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- main ---

def timed_search(torch, fn, flush, stream, steps):
    """Mean device milliseconds of fn() over `steps` calls (L2 flushed before
    each, CUDA events on the search's stream) and the last call's stats."""
    ts, st = [], None
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, st = fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts), st


def extra_rows(asci, torch, w, dets, cf, h1d, erid, ec, E0, flush, stream, args):
    import workloads as W
    rows = []
    steps = max(3, min(args.steps, 5))

    def add(label, ms, st, **extra):
        rows.append(dict(row=label, ms_per_step=round(ms, 3),
                         value=st.generated / (ms / 1e3), unit=UNIT, surviving=st.surviving,
                         unique=st.unique, **extra))

    fn = lambda: asci.search(dets, cf, E0, h1d, erid, ec, w.C, w.N, eps=1e-10)
    fn()
    ms, st = timed_search(torch, fn, flush, stream, steps)
    add(f"{w.name} eps=1e-10", ms, st)
    for name, prec in (("fp32_fp64acc", asci.FP32_INT_FP64_ACC), ("fp32_comp", asci.FP32_INT_COMP_ACC)):
        fn = lambda prec=prec: asci.search(dets, cf, E0, h1d, erid, ec, w.C, w.N, precision=prec)
        fn()
        ms, st = timed_search(torch, fn, flush, stream, steps)
        add(f"{w.name} precision={name}", ms, st)
    dev = dets.device
    for name in ("hubbard_8e8o", "random_16e16o"):
        if name not in W.WORKLOADS or name == w.name:
            continue
        ww = W.WORKLOADS[name]
        h1, eri, ec2 = ww.integrals()
        if ww.kind == "hubbard":  # the 100-determinant CI start of the (8e,8o) ring
            with open(os.path.join(ROOT, "tests", "golden", "hubbard_8e8o_psi.json")) as f:
                g = json.load(f)
            A, B, c, E02 = g["alpha"], g["beta"], g["c"], float(g["E0"])
        else:
            A, B, c = ww.psi()
            E02 = W.stored_e0(name)
        np_ = __import__("numpy")
        d = torch.tensor(np_.stack([np_.asarray(A, dtype=np_.uint64),
                                    np_.asarray(B, dtype=np_.uint64)], 1).astype("int64"),
                         device=dev)
        cc, hh, ee = (torch.tensor(np_.asarray(x, dtype=np_.float64), device=dev)
                      for x in (c, h1, eri))
        fn = lambda: asci.search(d, cc, E02, hh, ee, ec2, ww.C, ww.N)
        fn()
        ms, st = timed_search(torch, fn, flush, stream, max(steps, 5))
        add(name, ms, st, C=ww.C, N=ww.N, ndets=ww.ndets)
    return rows


def run_batched(args):
    """Many independent small searches (512 uneven systems): searches/s with the
    tuned number of concurrent streams and batch cap (tune_batched), against
    the same searches one at a time."""
    import numpy as np
    import torch
    import paper_2303_05688_gb300 as asci
    import workloads as W
    count = 512
    gen = W.batched_systems(count)
    dev = torch.device("cuda", 0)
    systems = []
    for sy in gen:
        d = torch.tensor(np.stack([sy["alpha"], sy["beta"]], 1).astype(np.int64), device=dev)
        h1 = torch.tensor(sy["h1"], device=dev)
        eri = torch.tensor(sy["eri"], device=dev)
        # E0 below the reference determinant's diagonal (an input of the search)
        dg = asci.diagonal(h1, eri, sy["ecore"], d[:1])
        E0 = float(dg.cpu()[0]) - 1.0
        systems.append(dict(dets=d, coeffs=torch.tensor(sy["c"], device=dev), E0=E0, h1=h1,
                            eri=eri, ecore=sy["ecore"], C=sy["C"], N=sy["N"]))
    prec = {"fp64": asci.FP64, "fp32_fp64acc": asci.FP32_INT_FP64_ACC,
            "fp32_comp": asci.FP32_INT_COMP_ACC}[args.precision]
    tuned = asci.tune_batched(systems, precision=prec)
    streams, bcap = tuned["streams"], tuned["max_batch_pairs"]
    for _ in range(max(args.warmup, 1)):
        asci.search_many(systems[:32], streams=streams, precision=prec, max_batch_pairs=bcap)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = asci.search_many(systems, streams=streams, precision=prec, max_batch_pairs=bcap)
    torch.cuda.synchronize()
    t_many = time.perf_counter() - t0
    t0 = time.perf_counter()
    for sy in systems:
        asci.search(sy["dets"], sy["coeffs"], sy["E0"], sy["h1"], sy["eri"], sy["ecore"],
                    sy["C"], sy["N"], precision=prec)
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    pairs = sum(st.generated for _, _, st in res)
    print(json.dumps({
        "metric": "batched ASCI searches/s (512 uneven systems, (8e,8o) to (20e,20o))",
        "value": count / t_many, "unit": "searches/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f64" if prec == asci.FP64 else "f32+f64",
        "data": "synthetic", "streams": streams, "max_batch_pairs": bcap,
        "serial": count / t_serial,
        "speedup_vs_serial": t_serial / t_many, "excitations_per_s": pairs / t_many,
        "config": {"workload": "batched512", "systems": count, "pairs": pairs}}), flush=True)
    return 0


def run_served(args):
    """Continuous-batching server: Poisson arrivals of search requests over
    resident systems from (8e,8o) to (24e,30o); p50/p99 latency and searches/s
    at 0.8 of the measured capacity, against the same requests one at a time
    in FP64, and the capacity with FP32 integrals and products."""
    import numpy as np
    import torch
    import paper_2303_05688_gb300 as asci
    from paper_2303_05688_gb300.serve import Server
    import workloads as W
    asci.load()
    rng = np.random.default_rng(11)
    reqs, resident = [], []
    for sy in W.batched_systems(24, seed=5000):
        resident.append((sy["name"], sy["alpha"], sy["beta"], sy["c"], sy["h1"], sy["eri"],
                         sy["ecore"], None))
        reqs.append((sy["name"], sy["C"], sy["N"], 0.9 / 24))
    for name, C, N, p in (("random_16e16o", 10000, 100000, 0.08),
                          ("random_24e30o", 20000, 10 ** 7, 0.02)):
        w, h1, eri, ec, A, B, c, E0, _ = load_workload(name)
        resident.append((name, A, B, c, h1, eri, ec, E0))
        reqs.append((name, C, N, p))
    probs = np.array([r[3] for r in reqs])
    picks = rng.choice(len(reqs), size=240, p=probs / probs.sum())
    stream_reqs = [reqs[i][:3] for i in picks]
    dev = torch.device("cuda", 0)
    slots = 8
    free, _ = torch.cuda.mem_get_info()
    budget = free // 2
    bp = int(min(1 << 29, budget // slots // 40))

    def serve(prec, arrivals=None):
        lat = []
        with Server(slots=slots, budget=budget) as srv:
            for name, A, B, c, h1, eri, ec, E0 in resident:
                d = torch.tensor(np.stack([A, B], 1).astype(np.int64), device=dev)
                if E0 is None:
                    dg = asci.diagonal(torch.tensor(h1, device=dev), torch.tensor(eri, device=dev),
                                       ec, d[:1])
                    E0 = float(dg.cpu()[0]) - 1.0
                srv.register(name, d, c, E0, h1, eri, ec)
            for name, C, N in stream_reqs[:8]:  # warm-up
                srv.submit(name, C, N, precision=prec, batch_pairs=bp).result()
            t0 = time.perf_counter()
            futs = []
            for i, (name, C, N) in enumerate(stream_reqs):
                if arrivals is not None:
                    delay = t0 + arrivals[i] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                futs.append(srv.submit(name, C, N, precision=prec, batch_pairs=bp))
            for f in futs:
                lat.append(f.result()[3])
            t = time.perf_counter() - t0
        return len(stream_reqs) / t, np.array(lat), srv

    cap, _, _ = serve(asci.FP64)
    lam = 0.8 * cap
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(stream_reqs)))
    rate, lat, srv = serve(asci.FP64, arrivals)
    cap32, _, _ = serve(asci.FP32_INT_COMP_ACC)
    # the same requests one at a time, FP64
    sysd = {}
    for name, A, B, c, h1, eri, ec, E0 in resident:
        d = torch.tensor(np.stack([A, B], 1).astype(np.int64), device=dev)
        h1d, ed = torch.tensor(h1, device=dev), torch.tensor(eri, device=dev)
        if E0 is None:
            E0 = float(asci.diagonal(h1d, ed, ec, d[:1]).cpu()[0]) - 1.0
        sysd[name] = (d, torch.tensor(c, device=dev), E0, h1d, ed, ec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for name, C, N in stream_reqs:
        d, cc, E0, h1d, ed, ec = sysd[name]
        asci.search(d, cc, E0, h1d, ed, ec, C, N, max_batch_pairs=bp)
    torch.cuda.synchronize()
    serial = len(stream_reqs) / (time.perf_counter() - t0)
    print(json.dumps({
        "metric": "served ASCI search: p50/p99 latency and searches/s at 0.8 x capacity",
        "value": rate, "unit": "searches/s", "n_gpus": 1, "higher_is_better": True,
        "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
        "capacity_fp64": cap, "capacity_fp32_products": cap32, "serial_fp64": serial,
        "arrival_rate": lam, "slots": slots, "peak_running": srv.peak_running,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "served", "requests": len(stream_reqs),
                   "systems": [r[0] for r in reqs], "mix": "90% 24 small systems, "
                   "8% (16e,16o) C=1e4 N=1e5, 2% (24e,30o) C=2e4 N=1e7"}}), flush=True)
    return 0


def run_levels(args):
    """Constraint-level study (Sec. 2.2, Fig. 2-3 analogue) on the (24e,30o)
    workload: for each deepest refinement level (3, 4, 5, 6 and n_alpha) and
    batch cap, the number of batches, the largest batch against the mean, and
    the search time (mean of args.steps after args.warmup)."""
    import torch
    import paper_2303_05688_gb300 as asci
    w, h1, eri, ec, A, B, c, E0, np = load_workload("random_24e30o")
    dev = torch.device("cuda", 0)
    d = torch.tensor(np.stack([A, B], 1).astype(np.int64), device=dev)
    cf, h1d, ed = (torch.tensor(x, device=dev) for x in (c, h1, eri))
    rows = []
    for bmax in (1 << 24, 1 << 26, 1 << 29):
        for lvl in (3, 4, 5, 6, w.na):
            def one():
                return asci.search(d, cf, E0, h1d, ed, ec, w.C, w.N, max_batch_pairs=bmax,
                                   max_constraint_level=lvl)
            for _ in range(max(args.warmup, 1)):
                one()
            torch.cuda.synchronize()
            ts = []
            for _ in range(max(args.steps, 1)):
                t0 = time.perf_counter()
                _, _, st = one()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            mean_batch = st.generated / max(st.batches, 1)
            rows.append({"max_batch_pairs": bmax, "max_level": lvl, "level_used": st.max_level,
                         "batches": st.batches, "largest_batch": st.max_batch,
                         "largest_over_mean": st.max_batch / mean_batch,
                         "ms": 1e3 * statistics.mean(ts)})
    # Fig. 3 analogue: the work (pairs) of every constraint class per level,
    # from the item weights of the search's own planning step
    classes = []
    for lvl in (3, 4, 5, 6):
        cnt = asci.constraint_classes(d, cf, h1d, ed, ec, w.C, lvl).astype(np.float64)
        hist = {}
        for k in np.floor(np.log2(cnt)).astype(int).tolist():
            hist[k] = hist.get(k, 0) + 1
        classes.append({"level": lvl, "classes": int(len(cnt)), "pairs": int(cnt.sum()),
                        "largest": int(cnt.max()), "mean": float(cnt.mean()),
                        "largest_over_mean": float(cnt.max() / cnt.mean()),
                        "median": float(np.median(cnt)),
                        "share_of_largest_1pct": float(np.sort(cnt)[::-1][:max(1, len(cnt) // 100)]
                                                       .sum() / cnt.sum()),
                        "log2_histogram": {f"2^{k}": v for k, v in sorted(hist.items())}})
    print(json.dumps({"metric": "constraint-level study, (24e,30o)", "unit": "ms",
                      "data": "synthetic", "rows": rows, "classes": classes}), flush=True)
    return 0


def run_pt2(args):
    """ASCI-PT2 (the last step of Alg. 1) on the (24e,30o) workload (or
    --pt2-workload) with the search's core (1e5 determinants): every unique
    target outside psi (5.5e9) contributes num^2 / (E0 - H_ii).  Mean of
    args.steps calls after args.warmup, inputs resident; L2 flushed before
    each call."""
    import torch
    import numpy as np
    import paper_2303_05688_gb300 as asci
    w, h1, eri, ec, A, B, c, E0, _ = load_workload(args.pt2_workload)
    dev = torch.device("cuda", 0)
    d = torch.tensor(np.stack([A, B], 1).astype(np.int64), device=dev)
    cf, h1d, ed = (torch.tensor(x, device=dev) for x in (c, h1, eri))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 1)):
        asci.pt2(d, cf, E0, h1d, ed, ec, w.C)
    times = []
    for _ in range(max(args.steps, 1)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        val, st = asci.pt2(d, cf, E0, h1d, ed, ec, w.C)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    core = size_cpu_sample(w, args)
    cpu = oracle_pt2_rate(w, h1, eri, ec, A, B, c, E0, core)
    print(json.dumps({
        "metric": f"ASCI-PT2 scored excitations/s on {w.name}", "unit": "excitations/s",
        "value": st.generated / (ms / 1e3), "ms_per_step": ms, "higher_is_better": True,
        "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": "f64",
        "config": {"workload": f"{w.name} pt2", "C": w.C, "ndets": w.ndets,
                   "l2": "flushed (512 MB write) before each step"},
        "cpu_baseline": {"value": cpu, "unit": "excitations/s", "cores": 1, "kind": "oracle",
                         "sample": f"oracle PT2 with the top {core} of {w.C} core dets of "
                                   f"{w.name}, full psi for exclusion"},
        "e_pt2": val, "targets": st.unique - st.excluded, "generated": st.generated,
        "batches": st.batches, "stage_ms": {k: round(v, 3) for k, v in st.t_stage_ms.items()}}),
        flush=True)
    return 0


def run_loop(args):
    """The ASCI loop (Alg. 1) on the (16e,16o) workload: three steps from its
    psi (1e5 determinants) with the (1e4, 1e5) core and wavefunction sizes;
    per step the device times of the search, the Hamiltonian build (Sec. 2.3)
    and Davidson (Alg. 5).  Then, on the final space, the build's element
    rate and the sparse product timed alone (CUDA events, the kernel queued
    behind a sleep so that host work is not timed), against the HBM peak
    (bytes: 12 per stored element, 8 per row pointer, 16 per row for x and
    y)."""
    import torch
    import numpy as np
    import paper_2303_05688_gb300 as asci
    w, h1, eri, ec, A, B, c, E0, _ = load_workload("random_16e16o")
    dev = torch.device("cuda", 0)
    d = torch.tensor(np.stack([A, B], 1).astype(np.int64), device=dev)
    cf, h1d, ed = (torch.tensor(x, device=dev) for x in (c, h1, eri))
    kw = dict(ncdets=w.C, ntdets=w.N, etol=0.0, tol=1e-8)
    asci.asci_loop(d, cf, h1d, ed, ec, max_steps=1, **kw)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    od, oc, E, st = asci.asci_loop(d, cf, h1d, ed, ec, max_steps=3, **kw)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    H = asci.hamiltonian(od, h1d, ed, ec)
    n, nnz = od.shape[0], H[1].numel()
    times = []
    # a device-side spin keeps the stream busy while the host prepares the call,
    # so that the events time the kernel alone (torch's private helper; without
    # it the time includes the host work of the call)
    spin = getattr(torch.cuda, "_sleep", None)
    for _ in range(max(args.steps, 5)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if spin is not None:
            spin(2_000_000)
        e0.record()
        asci.spmv(H, oc)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    peak, peak_kind = peaks()
    spmv_ms = statistics.median(times)
    spmv_bytes = 12 * nnz + 8 * (n + 1) + 16 * n
    steps = []
    for k in range(len(st.energy)):
        m = st.ndets[k]
        steps.append({"energy": st.energy[k], "ndets": m, "new_dets": st.new_dets[k],
                      "nnz": st.nnz[k], "davidson_products": st.davidson_iters[k],
                      "search_ms": round(st.t_search_ms[k], 3),
                      "hamiltonian_ms": round(st.t_hamiltonian_ms[k], 3),
                      "davidson_ms": round(st.t_davidson_ms[k], 3),
                      "elements_per_s": st.nnz[k] / (st.t_hamiltonian_ms[k] / 1e3)})
    last = steps[-1]
    pairs = od.cpu().numpy().view(np.uint64)
    cpu_rows = oracle_rows_per_s(h1, eri, ec, pairs[:, 0].copy(), pairs[:, 1].copy())
    print(json.dumps({
        "metric": "ASCI loop step time at (16e,16o)", "unit": "ms",
        "value": round(1e3 * wall / len(steps), 3), "higher_is_better": False,
        "data": "synthetic", "dtype": "f64",
        "config": {"workload": "random_16e16o loop", "ncdets": w.C, "ntdets": w.N,
                   "start_ndets": w.ndets, "steps": len(steps)},
        "start_energy": st.start_energy, "final_energy": E, "steps": steps,
        # the build prunes the pair loop by beta-string groups, so its rate is
        # given per stored element and, for context, per pair of the full
        # double loop it stands in for (2 n^2 pairs: counting and filling)
        "hamiltonian": {"ms": last["hamiltonian_ms"], "nnz": last["nnz"],
                        "rows_per_s": last["ndets"] / (last["hamiltonian_ms"] / 1e3),
                        "elements_per_s": last["elements_per_s"],
                        "double_loop_pairs_per_s": 2.0 * last["ndets"] ** 2 / (
                            last["hamiltonian_ms"] / 1e3)},
        "cpu_baseline": {"value": cpu_rows, "unit": "Hamiltonian rows/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"oracle dense rows of 16 of the final space's {n} determinants"},
        "spmv_roofline": {"bound": "hbm", "achieved": spmv_bytes / (spmv_ms / 1e3) / 1e9,
                          "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                          "frac": spmv_bytes / (spmv_ms / 1e3) / 1e9 / peak,
                          "ms": spmv_ms, "bytes": spmv_bytes, "n": n, "nnz": nnz}}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "levels":
        return run_levels(args)
    if args.workload == "batched512":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "asci_loop":
        return run_loop(args)
    if args.workload == "pt2":
        return run_pt2(args)

    import torch
    import torch.distributed as dist
    import paper_2303_05688_gb300 as asci

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    prec = {"fp64": asci.FP64, "fp32_fp64acc": asci.FP32_INT_FP64_ACC,
            "fp32_comp": asci.FP32_INT_COMP_ACC}[args.precision]
    w, h1, eri, ec, A, B, c, E0, np = load_workload(args.workload)
    dev = torch.device("cuda", local)
    dets = torch.tensor(np.stack([A, B], 1).astype(np.int64), device=dev)
    cf = torch.tensor(c, device=dev)
    h1d = torch.tensor(h1, device=dev)
    erid = torch.tensor(eri, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    asci.load()

    sharded = args.sharded and world > 1

    Ccore = args.C or w.C
    kw = dict(eps=args.eps, precision=prec)
    if args.max_batch_pairs:
        kw["max_batch_pairs"] = args.max_batch_pairs

    def one(d=dets, cc=cf, hh=h1d, ee=erid):
        if sharded:
            return asci.sharded_search(d, cc, E0, hh, ee, ec, Ccore, w.N, **kw)
        return asci.search(d, cc, E0, hh, ee, ec, Ccore, w.N, **kw)

    for _ in range(args.warmup):
        flush.zero_()
        one()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    l0 = asci.launch_count()
    times, stats = [], None
    tiles_ms, tile_records, tile_launches = 0.0, 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, stats = one()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        # the tile kernel's own launches, timed by the library with CUDA events
        # on the search's stream
        tiles_ms += stats.t_stage_ms["tiles"]
        tile_records += stats.tile_records
        tile_launches += stats.tile_launches
    torch.cuda.synchronize()
    barrier()
    launches = asci.launch_count() - l0
    clk = clocks.stop()
    t_total = sum(times) / 1e3
    if world > 1:
        t = torch.tensor([t_total], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
    pairs = stats.generated
    if sharded:  # every rank's shard of one search: total pairs of the search
        pt = torch.tensor([pairs], device=dev, dtype=torch.int64)
        dist.all_reduce(pt)
        pairs = int(pt.item())
        value = pairs * args.steps / t_total
    else:
        value = world * pairs * args.steps / t_total

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hd = torch.tensor(np.stack([A, B], 1).astype(np.int64)).pin_memory()
        hc = torch.tensor(c).pin_memory()
        hh = torch.tensor(h1).pin_memory()
        he = torch.tensor(eri).pin_memory()
        one(hd, hc, hh, he)
        torch.cuda.synchronize()
        barrier()
        te = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            od, osc, _ = one(hd, hc, hh, he)
            te.append(time.perf_counter() - t0)
        t_e2e = sum(te)
        if world > 1:
            t = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        h2d = hd.numel() * 8 + hc.numel() * 8 + hh.numel() * 8 + he.numel() * 8
        d2h = len(od) * 16 + len(osc) * 8
        e2e = {"value": (1 if sharded else world) * pairs * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel, the on-chip tile kernel (k_cells): it
    # reads each staged pair once (16 bytes); achieved = algorithmic bytes per
    # launch / its mean launch time (CUDA events in the library, live)
    peak, peak_kind = peaks()
    ts = stats.t_stage_ms
    per_launch_s = tiles_ms / 1e3 / max(tile_launches, 1)
    bytes_per_launch = 16.0 * tile_records / max(tile_launches, 1)
    achieved = bytes_per_launch / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    per_rec = TILE_DRAM_BYTES_PER_RECORD.get(w.name)
    traffic = per_rec * tile_records / max(tile_launches, 1) if per_rec else None
    traffic_note = (f"{per_rec} DRAM bytes per staged pair from {TILE_DRAM_SOURCE}, scaled to "
                    "one launch" if per_rec else "no capture of the current kernel")
    # the search as a whole against its algorithmic floor,
    # B_alg = 32 P + 24 C + 16 |psi| + 32 U + 16 N bytes
    b_alg = (32 * stats.surviving + 24 * stats.ncore + 16 * w.ndets + 32 * stats.unique
             + 16 * stats.selected)
    t_search = statistics.mean(times) / 1e3
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_note,
                "kernel": "k_cells (on-chip hash reduction of staged pairs)",
                "peak_kind": peak_kind, "launches_per_step": tile_launches / args.steps,
                "alg_bytes_per_launch": bytes_per_launch, "ms_per_launch": per_launch_s * 1e3,
                "search": {"alg_bytes_per_step": b_alg, "achieved": b_alg / t_search / 1e9,
                           "frac": b_alg / t_search / 1e9 / peak},
                # the sort-and-accumulate rate: staged pairs reduced per second
                # of the on-chip tile kernel and the global-sort path together
                "accumulate_pairs_per_s": (stats.tile_records + stats.oversized_records) / max(
                    (ts["tiles"] + ts["oversized"]) / 1e3, 1e-12),
                # pairs of hash buckets that hot targets overfilled, and those of
                # them reduced on chip by the large tile kernel
                "oversized_records": stats.oversized_records,
                "big_tile_records": stats.big_tile_records,
                "stage_ms": {k: round(v, 3) for k, v in ts.items()}}

    # further measured rows (same inputs, device-resident, L2 flushed, CUDA
    # events): the paper's screen eps = 1e-10 (Sec. 3), the two FP32-integral
    # variants, and the two smaller configurations
    rows = None
    if not args.no_rows and world == 1 and not sharded:
        rows = extra_rows(asci, torch, w, dets, cf, h1d, erid, ec, E0, flush, stream, args)

    cpu = cpu1 = None
    if not args.no_cpu_baseline and world == 1:
        cores = host_cores()
        core = size_cpu_sample(w, args, cores)
        p, dt = cpu_sample(w, h1, eri, ec, A, B, c, E0, core, np, cores)
        cpu = {"value": p / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"all-core oracle ({cores} threads) on the top {core} of {Ccore} core dets "
                         f"of {w.name} ({p} excitations, {dt:.1f} s), full psi for exclusion"}
        core1 = size_cpu_sample(w, args)
        p1, dt1 = cpu_sample(w, h1, eri, ec, A, B, c, E0, core1, np)
        cpu1 = {"value": p1 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"single-core oracle on the top {core1} of {w.C} core dets of {w.name} "
                          f"({p1} excitations, {dt1:.1f} s), full psi for exclusion"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f64" if prec == asci.FP64 else "f32+f64", "data": "synthetic",
        "config": {"workload": w.name, "norb": w.norb, "nelec": [w.na, w.nb], "ndets": w.ndets,
                   "C": Ccore, "N": w.N, "eps": args.eps, "precision": args.precision,
                   "excitations_per_step": pairs, "unique_per_step": stats.unique,
                   "batches": stats.batches, "l2": "flushed (512 MB write) before each step",
                   "parallelism": (f"constraint shards x{world}" if sharded
                                   else f"replicas x{world}")},
        "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
        "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_1core": cpu1, "rows": rows,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
