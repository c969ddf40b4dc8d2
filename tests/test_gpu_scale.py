"""Parity at the full sizes of the labelled workloads, in the launch
configurations the benchmark uses:

* R-MAT scale 24 (16.7M vertices, ~5e8 directed entries), 16 Zipf labels,
  random-walk queries of 8, 16, 24 and 32 vertices, half sparse (walk tree
  plus 1-2 edges) and half dense (induced), anchored at their source vertex
  and kept by the resampling rule: counts and hashes against the oracle.
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


def test_rmat24_zipf16_walk_queries(eng):
    # anchored random-walk queries of 8, 16, 24 and 32 vertices, dense and
    # sparse, kept by the resampling rule; each count and hash against the
    # oracle's count over the same one-vertex root slice
    from paper_2604_10601_gb300 import workload
    g = _labelled(24, 16, 3)
    G = eng.load_graph(g.rowptr, g.col, g.labels, 16)
    sizes = [8, 16, 24, 32] * 4
    dense = ([True] * 4 + [False] * 4) * 2
    cand = gg.walk_query_set(g, sizes, dense, seed=17)
    kept, _ = workload.select_bounded(eng, G, cand, workload.anchored_ranges(cand), keep=1 << 25)
    checked = 0
    for i in kept:
        q = cand[i]
        a = int(q.source[0])
        try:
            ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(0, a, a + 1),
                          max_steps=5 * 10 ** 7)
        except O.OracleError:
            continue
        Q = eng.query(q.k, q.edges, q.labels)
        Q.order_greedy(G, root=0)
        r = eng.count(G, Q, want_hash=True, root_range=(a, a + 1), time_cap_s=120)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), q.name
        assert eng.count(G, Q, root_range=(a, a + 1), time_cap_s=120)["count"] == ref["count"]
        assert r["count"] >= 1  # the walk's own vertices are an embedding
        checked += 1
        Q.free()
    assert checked >= 4, (len(kept), checked)
    G.free()


def test_rmat22_zipf32_batch_of_64_against_oracle(eng):
    g = _labelled(22, 32, 1)
    G = eng.load_graph(g.rowptr, g.col, g.labels, 32)
    from paper_2604_10601_gb300 import workload
    rng = np.random.default_rng(64)
    cand = gg.walk_query_set(g, [int(x) for x in rng.integers(4, 33, size=256)], [True] * 256, seed=64)
    kept, _ = workload.select_bounded(eng, G, cand, workload.anchored_ranges(cand), keep=1 << 24)
    qs = [cand[i] for i in kept][:64]
    assert len(qs) >= 16
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
