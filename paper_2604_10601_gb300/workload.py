"""Query-set helpers for the labelled random-walk workloads.

Random-walk queries (Sec. 6.1, Query Sets) on power-law graphs with skewed
labels can have astronomically many embeddings even when anchored at one
data vertex (a star around a hub of a frequent label). The paper handles
such queries with time limits and reports them as unsolved (Sec. 6.1,
Metrics). For query sets whose every count is exact, this module applies a
deterministic resampling rule instead: a query is kept when its count needs
at most `keep` partial matches in total (the sum of the per-level counts the
engine logs: the size of its search tree). The check runs the engine with a
work cap of 2 x keep candidate checks (sgm_opts.work_cap) and reads the
per-level counts of the completed run, which do not depend on timing or
scheduling.
"""
from __future__ import annotations

from . import sgm


def anchored_ranges(queries):
    """Root range of one data vertex per query: the walk's source vertex for query vertex 0."""
    return [(int(q.source[0]), int(q.source[0]) + 1) for q in queries]


def select_bounded(engine, graph, queries, root_ranges=None, keep=1 << 26):
    """(kept indices, rejected indices) of `queries` (graphgen.Query) under the
    rule above; root_ranges as in sgm_count_root_range (None = full ranges,
    else query vertex 0 is the root of the order)."""
    kept, rejected = [], []
    slack = 16384 * 8 * 4 * 152  # the work cap's reporting slack bound for any launch shape used here
    cap = max(2 * keep, keep + slack)
    for i, q in enumerate(queries):
        Q = engine.query(q.k, q.edges, q.labels)
        Q.order_greedy(graph, root=0 if root_ranges is not None else None)
        rr = None if root_ranges is None else root_ranges[i]
        try:
            r = engine.count(graph, Q, root_range=rr, work_cap=cap)
            work = int(r["level_counts"][:q.k].astype(object).sum())
            (kept if work <= keep else rejected).append(i)
        except sgm.SgmError as e:
            if e.status != sgm.SGM_E_WORK_CAP:
                raise
            rejected.append(i)
        finally:
            Q.free()
    return kept, rejected
