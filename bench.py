#!/usr/bin/env python3
"""Benchmark: exact subgraph counting on an R-MAT scale-20 graph.

Workload (one step = the whole query set, one query per launch, rule-based
greedy order, exact uint64 counts): R-MAT scale 20, edge factor 16,
(a, b, c) = (0.57, 0.19, 0.19), symmetrised, self-loops and duplicates
removed (31.4M directed CSR entries), unlabelled; queries K4, K5, C4, P5 and
the 6-vertex house with a diagonal, in both readings of that name (house5d:
5 vertices, 7 edges; house6d: 6 vertices, 8 edges).

metric: matches/s = embeddings counted over the step / step time (device
time, graph resident in HBM); ms_per_step is the query-set time.
e2e: the same metric through the public API from pinned host CSR arrays,
with the graph upload, table build and the read-back of the counts inside
the timed region.

--impl reference times the CPU oracle (single thread, as it stands) on a
bounded sample of the same workload (root slices), with the same metric.
Multi-GPU (--gpus N under torchrun): the root candidates of every query are
split into N contiguous vertex ranges, one per rank; counts are summed for
the report only (no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

QUERIES = ["K4", "K5", "C4", "P5", "house5d", "house6d"]
WORKLOAD = "rmat20_ef16_unlabelled_6q"
L2_BYTES = 129 * 1024 * 1024


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ["match_kernels.cu", "sgm_device.cuh", "sgm_internal.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2604_10601_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _ncu_traffic_per_launch():
    """DRAM bytes per extend_kernel launch from the committed ncu summary, or
    None when that summary was taken on another version of the kernel."""
    p = os.path.join(ROOT, "profiles", "extend_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_hash") != _kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_gpu{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _workload_graph():
    import graphgen as gg
    return gg.rmat_graph(20, 16, 0.57, 0.19, 0.19, seed=1)


def _shard(n, world, rank):
    return rank * n // world, (rank + 1) * n // world


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import graphgen as gg
    from paper_2604_10601_gb300 import Engine
    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = _workload_graph()
    lo, hi = _shard(g.n, world, rank)
    eng = Engine(local)
    # resident graph (device-timed arm)
    G = eng.load_graph(g.rowptr, g.col)
    qs = []
    for name in QUERIES:
        p = gg.pattern(name)
        Q = eng.query(p.k, p.edges)
        Q.order_greedy(G)
        qs.append((name, Q))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(G):
        tot, alg_bytes, ext_ms, launches = 0, 0.0, 0.0, 0
        per = {}
        for name, Q in qs:
            r = eng.count(G, Q, root_range=(lo, hi))
            s = r["stats"]
            tot += r["count"]
            per[name] = r["count"]
            alg_bytes += 4.0 * s["list_elems"] + 32.0 * (s["search_probes"] + s["bitmap_probes"]) + \
                12.0 * s["task_groups"]
            ext_ms += s["ms_search"]
            launches += s["launches"] if "launches" in s else 0
        return tot, per, alg_bytes, ext_ms, launches

    for _ in range(args.warmup):
        step(G)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, alg_total, ext_total, launches_total, counts = [], 0.0, 0.0, 0, None
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            tot, per, ab, em, nl = step(G)
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            alg_total += ab
            ext_total += em
            launches_total += nl
            counts = per
    clocks = clk.summary()
    ms = sum(times) / len(times)
    t_max = torch.tensor([ms], dtype=torch.float64, device=dev)
    tot_t = torch.tensor([sum(counts.values())], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot_t, op=dist.ReduceOp.SUM)
    ms_step = float(t_max.item())
    total_matches = float(tot_t.item())

    # end-to-end: pinned host CSR -> engine -> counts back on the host
    rp_h = torch.from_numpy(g.rowptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    e2e_times = []
    for i in range(max(1, min(args.steps, 3)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ge = eng.load_graph(rp_h.numpy(), col_h.numpy())
        e_tot = 0
        for name, Q in qs:
            e_tot += eng.count(Ge, Q, root_range=(lo, hi))["count"]
        Ge.free()
        t1 = time.perf_counter()
        if i > 0:
            e2e_times.append((t1 - t0) * 1e3)
    e2e_ms = sum(e2e_times) / len(e2e_times)
    e2e_t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_ms = float(e2e_t.item())

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    hbm, peak_kind = _peaks()
    achieved = (alg_total / (ext_total / 1e3)) / 1e9 if ext_total > 0 else 0.0
    traffic = _ncu_traffic_per_launch()
    h2d = g.rowptr.nbytes + g.col.nbytes + sum(8 * p.k for p in map(gg.pattern, QUERIES))
    out = {
        "metric": "matches/s", "value": total_matches / (ms_step / 1e3), "unit": "matches/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "graph": "rmat scale 20, ef 16, a=.57 b=.19 c=.19, seed 1",
                   "n": g.n, "directed_entries": g.nnz, "queries": QUERIES, "order": "greedy",
                   "counts": counts, "l2": "flushed before every timed step (2x L2 write)",
                   "parallelism": f"root-range shards x{world}"},
        "query_set_ms": ms_step,
        "e2e": {"value": total_matches / (e2e_ms / 1e3), "unit": "matches/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8 * len(QUERIES) * 34},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": "extend_kernel"},
        "gpu_launches": launches_total // max(1, args.steps) * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# --------------------------------------------------------------------------
def _oracle_sample(budget_s, g=None):
    """The oracle on root slices of every query, growing the slice until the
    budget is spent; returns (matches, seconds, description)."""
    import graphgen as gg
    import oracle as O
    g = g if g is not None else _workload_graph()
    per_q = budget_s / len(QUERIES)
    tot_m, tot_s, desc = 0, 0.0, []
    for name in QUERIES:
        p = gg.pattern(name)
        own = O.match(np.zeros(2, np.int64), np.zeros(0, np.int32), None, p.k, p.edges)["order"]
        root = int(own[0])
        # start at the top of the id range (low degrees) and grow downwards
        width, lo, spent, m = 64, g.n, 0.0, 0
        while spent < per_q and lo > 0:
            a = max(0, lo - width)
            t0 = time.perf_counter()
            try:
                r = O.match(g.rowptr, g.col, None, p.k, p.edges, root=(root, a, lo), max_steps=2 * 10 ** 9)
            except O.OracleError:
                break
            dt = time.perf_counter() - t0
            spent += dt
            m += r["count"]
            lo = a
            width *= 2
        tot_m += m
        tot_s += spent
        desc.append(f"{name}: M[{root}] in [{lo},{g.n}) {m} matches {spent:.1f}s")
    return tot_m, tot_s, "; ".join(desc)


def cpu_baseline(budget_s):
    m, s, desc = _oracle_sample(budget_s)
    return {"value": m / s if s > 0 else 0.0, "unit": "matches/s", "cores": 1, "kind": "oracle",
            "sample": f"single-thread oracle on root slices of the same graph and queries ({desc})"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    g = _workload_graph()
    budget = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        _oracle_sample(budget, g)
    tm, ts, desc = 0, 0.0, ""
    for _ in range(args.steps):
        m, s, desc = _oracle_sample(budget, g)
        tm += m
        ts += s
    v = tm / ts if ts > 0 else 0.0
    out = {"impl": "reference", "metric": "matches/s", "value": v, "unit": "matches/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * ts / max(1, args.steps),
           "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "queries": QUERIES, "sample": "root slices"},
           "cpu_baseline": {"value": v, "unit": "matches/s", "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "matches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
