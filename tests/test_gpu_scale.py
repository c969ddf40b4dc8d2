"""Parity at the full sizes of the labelled workloads, in the launch
configurations the benchmark uses:

* R-MAT scale 24 (16.7M vertices, ~5e8 directed entries), 16 Zipf labels,
  random-walk queries of 8, 16, 24 and 32 vertices, half sparse (walk tree
  plus 1-2 edges) and half dense (induced): each query's count over the
  root slice holding its source vertex against the oracle; the full count
  where the oracle finishes within its step budget.
* R-MAT scale 22, 32 Zipf labels, 64 seeded walk queries of 4-32 vertices,
  anchored at their source vertex, in one batched launch: every count and
  hash against the oracle (or, where the oracle's step budget runs out,
  against the plain engine)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine
    return Engine(0)


def _labelled(scale, labels, seed):
    g = gg.rmat_graph(scale, 16, 0.57, 0.19, 0.19, seed=seed)
    g.labels = gg.labels_zipf(g.n, labels, 1.0, seed + 1)
    g.num_labels = labels
    return g


def _check_query(eng, g, G, q, budget):
    """Full count against the oracle when it finishes, else the source slice."""
    Q = eng.query(q.k, q.edges, q.labels)
    try:
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, max_steps=budget)
        r = eng.count(G, Q, want_hash=True, time_cap_s=120)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), q.name
        full = True
    except O.OracleError:
        v = int(q.source[0])
        Q.order_greedy(G, root=0)
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(0, v, v + 1), max_steps=budget)
        r = eng.count(G, Q, want_hash=True, root_range=(v, v + 1), time_cap_s=120)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), q.name
        assert eng.count(G, Q, root_range=(v, v + 1), time_cap_s=120)["count"] == ref["count"]
        full = False
    assert r["count"] >= 1  # the walk's own vertices are an embedding
    Q.free()
    return full


def test_rmat24_zipf16_walk_queries(eng):
    g = _labelled(24, 16, 3)
    G = eng.load_graph(g.rowptr, g.col, g.labels, 16)
    sizes = [8, 16, 24, 32] * 2
    dense = [True] * 4 + [False] * 4
    qs = gg.walk_query_set(g, sizes, dense, seed=17)
    fulls = [_check_query(eng, g, G, q, 5 * 10 ** 7) for q in qs]
    assert len(fulls) == 8
    G.free()


def test_rmat22_zipf32_batch_of_64_against_oracle(eng):
    g = _labelled(22, 32, 1)
    G = eng.load_graph(g.rowptr, g.col, g.labels, 32)
    rng = np.random.default_rng(64)
    qs = gg.walk_query_set(g, [int(x) for x in rng.integers(4, 33, size=64)], [True] * 64, seed=64)
    Qs = [eng.query(q.k, q.edges, q.labels) for q in qs]
    for Q in Qs:
        Q.order_greedy(G, root=0)
    ranges = [(int(q.source[0]), int(q.source[0]) + 1) for q in qs]
    r = eng.count_batch(G, Qs, want_hash=True, root_ranges=ranges, time_cap_s=120)
    for i, q in enumerate(qs):
        a = ranges[i][0]
        try:
            ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(0, a, a + 1),
                          max_steps=2 * 10 ** 7)
            assert (int(r["counts"][i]), int(r["hashes"][i])) == (ref["count"], ref["hash"]), q.name
        except O.OracleError:
            # too large for the oracle: the batched count equals the plain engine's
            assert int(r["counts"][i]) == eng.count(G, Qs[i], root_range=ranges[i], time_cap_s=120)["count"]
    G.free()
