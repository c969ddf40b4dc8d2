"""The rule-based greedy matching order (host side, no GPU), through the
host-only ABI call: hand-worked cases of each tie-break, and validity
(a connected permutation) on random queries."""
import numpy as np
import pytest

import graphgen as gg
from paper_2604_10601_gb300 import sgm


def _order(q, counts=None, root=-1):
    return [int(x) for x in sgm.sgm_query_greedy_order_host(q.k, q.edges, q.labels, counts, root)]


def test_hand_worked_orders():
    # K4: all ties, smallest ids first
    assert _order(gg.pattern("K4"), [100]) == [0, 1, 2, 3]
    # star: the centre (largest degree) first
    assert _order(gg.pattern("S3"), [100]) == [0, 1, 2, 3]
    # path 0-1-2-3: a middle vertex first (degree 2, smaller id); then 2, which
    # still has an unvisited neighbour, before 0
    assert _order(gg.pattern("P4"), [100]) == [1, 2, 0, 3]
    # tailed triangle: vertex 0 (degree 3), then the triangle before the tail
    assert _order(gg.pattern("tailed_triangle"), [10, 10, 10]) == [0, 1, 2, 3]
    # rarer label breaks a degree tie: C4 labelled (0, 1, 0, 1), label 1 rare
    c4 = gg.Query(4, [[0, 1], [1, 2], [2, 3], [3, 0]], [0, 1, 0, 1])
    assert _order(c4, [100, 3]) == [1, 0, 2, 3]
    assert _order(c4, [3, 100]) == [0, 1, 2, 3]
    # a fixed root
    assert _order(gg.pattern("P4"), [100], root=3) == [3, 2, 1, 0]


@pytest.mark.parametrize("seed", range(5))
def test_orders_are_connected_permutations(seed):
    rng = np.random.default_rng(900 + seed)
    for _ in range(20):
        k = int(rng.integers(2, 20))
        edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}
        for _ in range(int(rng.integers(0, k))):
            a, b = sorted(int(x) for x in rng.choice(k, 2, replace=False))
            edges.add((a, b))
        q = gg.Query(k, sorted(edges), rng.integers(0, 4, size=k).astype(np.int32))
        counts = rng.integers(1, 1000, size=4)
        for root in (-1, int(rng.integers(0, k))):
            phi = _order(q, counts, root)
            assert sorted(phi) == list(range(k))
            if root >= 0:
                assert phi[0] == root
            adj = [set() for _ in range(k)]
            for a, b in edges:
                adj[a].add(b)
                adj[b].add(a)
            assert all(adj[phi[i]] & set(phi[:i]) for i in range(1, k))


def test_disconnected_query_is_rejected():
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_query_greedy_order_host(4, [[0, 1], [2, 3]])
    assert ei.value.status == sgm.SGM_E_QUERY_DISCONNECTED
