"""Batched execution (many queries in one captured persistent launch)
against separate runs and the oracle, through the C ABI: counts and hashes
bit-exact, on labelled random-walk queries of uneven sizes and on the
unlabelled patterns; replays of the captured graph give the same results."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine
    return Engine(0)


@pytest.fixture(scope="module")
def labelled():
    g = gg.rmat_graph(12, 8, seed=41)
    g.labels = gg.labels_zipf(g.n, 8, 1.0, 41)
    g.num_labels = 8
    return g


def _walk_queries(g, n, seed, kmin=4, kmax=12):
    # induced (dense) random-walk queries: the batched workload's query shape
    rng = np.random.default_rng(seed)
    sizes = [int(x) for x in rng.integers(kmin, kmax + 1, size=n)]
    return gg.walk_query_set(g, sizes, [True] * n, seed=seed)


def test_batch_matches_separate_runs_and_oracle(eng, labelled):
    # anchored queries: query vertex 0 fixed to the walk's source vertex
    from paper_2604_10601_gb300 import workload
    g = labelled
    G = eng.load_graph(g.rowptr, g.col, g.labels, 8)
    cand = _walk_queries(g, 80, 5)
    kept, _ = workload.select_bounded(eng, G, cand, workload.anchored_ranges(cand), keep=1 << 22)
    qs = [cand[i] for i in kept][:40]
    assert len(qs) >= 20
    Qs = [eng.query(q.k, q.edges, q.labels) for q in qs]
    for Q in Qs:
        Q.order_greedy(G, root=0)
    ranges = [(int(q.source[0]), int(q.source[0]) + 1) for q in qs]
    sep = [eng.count(G, Q, want_hash=True, root_range=rr, time_cap_s=60) for Q, rr in zip(Qs, ranges)]
    b = eng.batch(G, Qs, want_hash=True, root_ranges=ranges, time_cap_s=120)
    r1 = b.run()
    r2 = b.run()
    for i in range(len(qs)):
        assert (int(r1["counts"][i]), int(r1["hashes"][i])) == (sep[i]["count"], sep[i]["hash"]), qs[i].name
    assert np.array_equal(r1["counts"], r2["counts"]) and np.array_equal(r1["hashes"], r2["hashes"])
    assert not r1["statuses"].any()
    b.free()
    # count-only batch, other launch shapes
    for kw in [dict(), dict(chunk_words=1, warps_per_block=4), dict(chunk_words=64, split_min=0),
               dict(chunk_words=2, split_min=8, sym_break=0)]:
        r = eng.count_batch(G, Qs, root_ranges=ranges, **kw, time_cap_s=120)
        assert [int(x) for x in r["counts"]] == [s["count"] for s in sep], kw
    for q, s, rr in list(zip(qs, sep, ranges))[:12]:
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(0, rr[0], rr[1]), max_steps=10 ** 8)
        assert (s["count"], s["hash"]) == (ref["count"], ref["hash"]), q.name



def test_batch_unlabelled_patterns_and_tiny_queries(eng):
    g = gg.rmat_graph(10, 2, seed=11)
    G = eng.load_graph(g.rowptr, g.col)
    names = ["K3", "K4", "C4", "P3", "P4", "S2", "S3", "house5d", "house6d", "C5"]
    qs = [gg.pattern(nm) for nm in names]
    qs.append(gg.Query(1, np.zeros((0, 2), np.int32)))
    qs.append(gg.Query(2, [[0, 1]]))
    Qs = [eng.query(q.k, q.edges, q.labels) for q in qs]
    for want_hash in (False, True):
        r = eng.count_batch(G, Qs, want_hash=want_hash, time_cap_s=120)
        for i, q in enumerate(qs):
            ref = O.match(g.rowptr, g.col, None, q.k, q.edges)
            assert int(r["counts"][i]) == ref["count"], q.name
            if want_hash:
                assert int(r["hashes"][i]) == ref["hash"], q.name
    # root ranges of several words with ragged ends, against the oracle's slices
    wide = [(37 * i, 37 * i + 200 + 13 * i) for i in range(len(qs))]
    for Q in Qs:
        Q.order_greedy(G, root=0)
    rb = eng.count_batch(G, Qs, want_hash=True, root_ranges=wide, time_cap_s=120)
    for i, (q, rr) in enumerate(zip(qs, wide)):
        ref = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(0, rr[0], rr[1]))
        assert (int(rb["counts"][i]), int(rb["hashes"][i])) == (ref["count"], ref["hash"]), q.name


def test_empty_batch_and_errors(eng, labelled):
    from paper_2604_10601_gb300 import sgm
    g = labelled
    G = eng.load_graph(g.rowptr, g.col, g.labels, 8)
    r = eng.count_batch(G, [])
    assert len(r["counts"]) == 0
    Q = eng.query(2, [[0, 1]], [0, 99])
    with pytest.raises(sgm.SgmError) as ei:
        eng.count_batch(G, [Q])
    assert ei.value.status == sgm.SGM_E_LABEL_RANGE
