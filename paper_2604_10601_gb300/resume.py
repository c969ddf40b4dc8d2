"""Checkpointed counting over root slices.

Root slices partition the embeddings of a query (sgm_count_root_range: the
slices of a partition of [0, n) sum to the full count and hash), so a long
count can run slice by slice and resume after an interruption. The state is
a small JSON file, rewritten atomically after every slice: the slices still
to run, and the count and hash (mod 2^64) of the finished ones.
"""
from __future__ import annotations

import json
import os

from .shard import MASK64


def plan_slices(n: int, parts: int) -> list[tuple[int, int]]:
    """`parts` contiguous root ranges covering [0, n)."""
    parts = max(1, int(parts))
    cuts = [i * n // parts for i in range(parts + 1)]
    return [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def _save(path: str, state: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(state, f)
    os.replace(tmp, path)


def resumable_count(count_slice, n: int, parts: int, state_path: str, max_slices=None) -> dict:
    """Counts over root slices of [0, n), resuming from `state_path` when it
    exists. count_slice(lo, hi) returns (count, hash) of one slice (for
    example a call of Engine.count with root_range=(lo, hi)). Stops after
    `max_slices` slices of this call (None = all); returns the state:
    {"n", "slices" (left), "count", "hash", "done"}."""
    if os.path.exists(state_path):
        with open(state_path) as f:
            state = json.load(f)
        if state.get("n") != n:
            raise ValueError(f"state file {state_path} is for n = {state.get('n')}, not {n}")
    else:
        state = {"n": n, "slices": [list(s) for s in plan_slices(n, parts)], "count": 0, "hash": 0, "done": 0}
        _save(state_path, state)
    ran = 0
    while state["slices"] and (max_slices is None or ran < max_slices):
        lo, hi = state["slices"][0]
        c, h = count_slice(lo, hi)
        state["count"] += int(c)
        state["hash"] = (state["hash"] + int(h)) & MASK64
        state["slices"].pop(0)
        state["done"] += 1
        _save(state_path, state)
        ran += 1
    return state
