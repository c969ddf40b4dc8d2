"""Per-query run records as JSON lines.

One record per engine call: the query's name and root range, its count,
hash and per-level partial-match counts (the cost model's training data),
the phase times, and the extension kernel's work counters turned into the
quantities the benchmark reports: intersected elements (local-list
elements streamed through membership tests), algorithmic bytes (the
engine's own count: 8 B per backward neighbour of a task group, 4 B per
list element, per membership test 32 B into a hub bitmap or the cheaper of
streaming and searching the sorted row), the probe-sector bytes of the
coarser model kept for comparison (4 B per list element, one 32-B sector
per probe, 12 B per task group), the idle rate (empty lane slots per
scatter round, Sec. 2.3) and the steals.
"""
from __future__ import annotations

import json

import numpy as np


def alg_bytes(stats) -> float:
    """Algorithmic bytes of one call: the engine's own count (sgm_stats.alg_bytes)."""
    return float(stats["alg_bytes"])


def probe_sector_bytes(stats) -> float:
    """The coarser byte model: 4 B per list element, one 32-B sector per
    membership probe (every bisection step), 12 B per task group."""
    return (4.0 * stats["list_elems"] + 32.0 * (stats["search_probes"] + stats["bitmap_probes"])
            + 12.0 * stats["task_groups"])


def record(name, result, root_range=None, **extra) -> dict:
    """A JSON-ready record of one count result (Engine.count's dict)."""
    st = result["stats"]
    lc = result.get("level_counts")
    rounds = int(st["scatter_rounds"])
    rec = {
        "query": name,
        "root_range": None if root_range is None else [int(root_range[0]), int(root_range[1])],
        "count": int(result["count"]),
        "hash": None if result.get("hash") is None else int(result["hash"]),
        "level_counts": None if lc is None else [int(x) for x in np.asarray(lc).tolist()],
        "ms_filter": float(st["ms_filter"]), "ms_init": float(st["ms_init"]), "ms_search": float(st["ms_search"]),
        "init_depth": int(st["init_depth"]), "pool_size": int(st["pool_size"]),
        "intersected_elements": int(st["list_elems"]),
        "membership_probes": int(st["search_probes"]) + int(st["bitmap_probes"]),
        "task_groups": int(st["task_groups"]),
        "alg_bytes": alg_bytes(st),
        "probe_sector_bytes": probe_sector_bytes(st),
        "idle_rate": (int(st["idle_lanes"]) / (32.0 * rounds)) if rounds else None,
        "steals": int(st["steals"]), "launches": int(st["launches"]), "aut_size": int(st["aut_size"]),
    }
    rec.update(extra)
    return rec


def append(path: str, rec: dict) -> None:
    """Appends one record as a line of JSON."""
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def read(path: str) -> list[dict]:
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]
