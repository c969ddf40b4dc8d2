"""Autotuner for the launch parameters of batched and single-query runs.

It times the engine's own runs (device time from the CUDA events libsgm
records) over a small grid of parameters and keeps the fastest setting:

  chunk_words      task granularity of batched runs (bitmap words of 32 root
                   candidates per initial task)
  warps_per_block  warps per block of the persistent extension kernel
  split_min        candidate-range length above which a warp offers half of
                   its range to idle warps (0: no work queue)
  pool_chunk       candidates per range task cut from the initial pool's long lists
  tau              initial-pool threshold of the breadth-first initialisation (Sec. 4.3)
  blocks_per_sm    resident blocks per SM (0: as many as fit)
  hub_min_deg      the intersection variant: vertices of at least this degree
                   answer membership tests from an adjacency bitmap, the others
                   by bisection of their sorted row (read when a graph loads)

Counts must agree across every setting (they are exact); a setting whose
counts differ raises. The result is a plain dict that can be saved as JSON
and passed back as keyword options.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np

from . import sgm

DEFAULT_BATCH_GRID = dict(chunk_words=[4], warps_per_block=[4, 8], split_min=[0, 16, 256], blocks_per_sm=[0])
DEFAULT_SINGLE_GRID = dict(warps_per_block=[4, 8], split_min=[64, 256, 1024], pool_chunk=[256, 1024], blocks_per_sm=[0],
                           tau=[10 ** 5, 10 ** 6])


def _grid(grid):
    keys = sorted(grid)
    for vals in itertools.product(*(grid[k] for k in keys)):
        yield dict(zip(keys, vals))


def tune_batch(engine, graph, queries, grid=None, repeats=2, time_cap_s=60.0, root_ranges=None) -> dict:
    """Best batched setting for `queries` (a list of sgm.Query) on `graph`."""
    grid = grid or DEFAULT_BATCH_GRID
    table, ref = [], None
    for kw in _grid(grid):
        b = engine.batch(graph, queries, root_ranges=root_ranges, time_cap_s=time_cap_s, **kw)
        times = []
        try:
            for _ in range(repeats):
                r = b.run(check=False)
                if r["status"] == sgm.SGM_E_TIME_CAP:
                    times = [float("inf")]  # this setting does not finish within the cap
                    break
                if r["status"] < 0:
                    raise sgm.SgmError(int(r["status"]), "sgm_batch_run")
                times.append(r["ms"])
                if ref is None:
                    ref = r["counts"].copy()
                elif not np.array_equal(ref, r["counts"]):
                    raise RuntimeError(f"counts differ under {kw}")
        finally:
            b.free()
        table.append(dict(kw, ms=float(min(times))))
    best = min(table, key=lambda row: row["ms"])
    if best["ms"] == float("inf"):
        raise RuntimeError("no setting of the grid finished within the time cap")
    return dict(best={k: v for k, v in best.items() if k != "ms"}, best_ms=best["ms"], table=table)


def tune_single(engine, graph, queries, grid=None, repeats=1, time_cap_s=60.0, root_ranges=None) -> dict:
    """Best setting of one-query-per-launch runs, by the summed device time."""
    grid = grid or DEFAULT_SINGLE_GRID
    table, ref = [], None
    for kw in _grid(grid):
        tot, counts = 0.0, []
        for i, Q in enumerate(queries):
            best = None
            rr = None if root_ranges is None else root_ranges[i]
            for _ in range(repeats):
                try:
                    r = engine.count(graph, Q, time_cap_s=time_cap_s, root_range=rr, **kw)
                except sgm.SgmError as e:
                    if e.status != sgm.SGM_E_TIME_CAP:
                        raise
                    best = float("inf")  # does not finish within the cap
                    break
                t = r["stats"]["ms_filter"] + r["stats"]["ms_init"] + r["stats"]["ms_search"]
                best = t if best is None else min(best, t)
            tot += best
            counts.append(r["count"] if best != float("inf") else None)
        if tot != float("inf"):
            if ref is None:
                ref = counts
            elif counts != ref:
                raise RuntimeError(f"counts differ under {kw}")
        table.append(dict(kw, ms=tot))
    best = min(table, key=lambda row: row["ms"])
    if best["ms"] == float("inf"):
        raise RuntimeError("no setting of the grid finished within the time cap")
    return dict(best={k: v for k, v in best.items() if k != "ms"}, best_ms=best["ms"], table=table)


DEFAULT_HUB_THRESHOLDS = [32, 128, 512, 4096, 1 << 30]  # the last one: no bitmaps, bisection only


def tune_hub_threshold(engine, rowptr, col, labels, num_labels, queries, root_ranges=None, thresholds=None,
                       repeats=1, time_cap_s=60.0, **count_opts) -> dict:
    """Best hub-bitmap degree threshold for one-query-per-launch runs of
    `queries` (sgm.Query objects registered on `engine`), by the summed
    device time. The graph is loaded once per threshold, since the engine
    reads SGM_HUB_MIN_DEG when a graph loads; the variable is restored
    afterwards."""
    thresholds = thresholds or DEFAULT_HUB_THRESHOLDS
    table, ref = [], None
    old = os.environ.get("SGM_HUB_MIN_DEG")
    try:
        for t in thresholds:
            os.environ["SGM_HUB_MIN_DEG"] = str(int(t))
            G = engine.load_graph(rowptr, col, labels, num_labels)
            tot, counts = 0.0, []
            try:
                hubs = int(G.info["hubs"])
                for i, Q in enumerate(queries):
                    rr = None if root_ranges is None else root_ranges[i]
                    best = None
                    for _ in range(repeats):
                        try:
                            r = engine.count(G, Q, time_cap_s=time_cap_s, root_range=rr, **count_opts)
                        except sgm.SgmError as e:
                            if e.status != sgm.SGM_E_TIME_CAP:
                                raise
                            best = float("inf")  # does not finish within the cap
                            break
                        st = r["stats"]
                        ms = st["ms_filter"] + st["ms_init"] + st["ms_search"]
                        best = ms if best is None else min(best, ms)
                    tot += best
                    counts.append(r["count"] if best != float("inf") else None)
            finally:
                G.free()
            if tot != float("inf"):
                if ref is None:
                    ref = counts
                elif counts != ref:
                    raise RuntimeError(f"counts differ under hub_min_deg={t}")
            table.append(dict(hub_min_deg=int(t), hubs=hubs, ms=tot))
    finally:
        if old is None:
            os.environ.pop("SGM_HUB_MIN_DEG", None)
        else:
            os.environ["SGM_HUB_MIN_DEG"] = old
    best = min(table, key=lambda row: row["ms"])
    if best["ms"] == float("inf"):
        raise RuntimeError("no threshold finished within the time cap")
    return dict(best={"hub_min_deg": best["hub_min_deg"]}, best_ms=best["ms"], table=table)


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)["best"]
