"""Checkpointed counting over root slices (host logic, no GPU): an
interrupted run resumed from its state file gives the oracle's full count
and hash, and the state file guards against a different graph."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from paper_2604_10601_gb300 import resume


def test_slices_cover_the_range():
    for n, parts in [(0, 3), (1, 4), (10, 3), (1000, 7)]:
        s = resume.plan_slices(n, parts)
        assert sum(b - a for a, b in s) == n
        assert all(s[i][1] == s[i + 1][0] for i in range(len(s) - 1))


def test_interrupted_count_resumes_to_the_full_result(tmp_path):
    g = gg.rmat_graph(10, 4, seed=5)
    q = gg.pattern("house5d")
    own = O.match(np.zeros(2, np.int64), np.zeros(0, np.int32), None, q.k, q.edges)["order"]
    root = int(own[0])

    def count_slice(lo, hi):
        r = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(root, lo, hi))
        return r["count"], r["hash"]

    path = str(tmp_path / "state.json")
    st = resume.resumable_count(count_slice, g.n, 9, path, max_slices=4)
    assert st["done"] == 4 and len(st["slices"]) == 5
    st = resume.resumable_count(count_slice, g.n, 9, path)  # resumed
    full = O.match(g.rowptr, g.col, None, q.k, q.edges)
    assert (st["count"], st["hash"]) == (full["count"], full["hash"])
    assert st["done"] == 9 and not st["slices"]
    with pytest.raises(ValueError):
        resume.resumable_count(count_slice, g.n + 1, 9, path)
