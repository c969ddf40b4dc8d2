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


def test_batch_size_classes_and_per_query_work_cap(eng, labelled):
    """Anchored walk queries of every size class (k = 2..32) in one batch;
    with a per-query work cap the hard ones stop as unsolved while every
    solved one equals its separate, uncapped run."""
    from paper_2604_10601_gb300 import sgm
    g = labelled
    G = eng.load_graph(g.rowptr, g.col, g.labels, 8)
    sizes = [2, 3, 4, 5, 6, 7, 8, 9, 12, 15, 16, 17, 20, 23, 24, 25, 28, 31, 32] * 2
    qs = gg.walk_query_set(g, sizes, [i % 2 == 0 for i in range(len(sizes))], seed=77)
    Qs = [eng.query(q.k, q.edges, q.labels) for q in qs]
    for Q in Qs:
        Q.order_greedy(G, root=0)
    ranges = [(int(q.source[0]), int(q.source[0]) + 1) for q in qs]
    # a small cap: every query whose search needs more than a few thousand
    # checks per warp stops, the small ones finish
    cap = 1 << 12
    b = eng.batch(G, Qs, root_ranges=ranges, work_cap=cap, time_cap_s=120)
    r = b.run(check=False)
    b.free()
    st = r["statuses"]
    assert set(int(x) for x in st) <= {0, sgm.SGM_E_WORK_CAP}
    solved = [i for i in range(len(qs)) if st[i] == 0]
    assert len(solved) >= 4 and len(solved) < len(qs)
    for i in solved:
        want = eng.count(G, Qs[i], root_range=ranges[i], time_cap_s=120)["count"]
        assert int(r["counts"][i]) == want, qs[i].name
        assert want >= 1  # the walk itself is an embedding
    for i in range(len(qs)):
        if st[i] != 0:
            assert int(r["counts"][i]) == 0
    # without a cap, the queries the resampling rule keeps match their separate runs
    from paper_2604_10601_gb300 import workload
    small, _ = workload.select_bounded(eng, G, qs, ranges, keep=1 << 22)
    rb = eng.count_batch(G, [Qs[i] for i in small], root_ranges=[ranges[i] for i in small], time_cap_s=120)
    for j, i in enumerate(small):
        assert int(rb["counts"][j]) == eng.count(G, Qs[i], root_range=ranges[i], time_cap_s=120)["count"]
    # hashes of the solved ones, against the oracle on a few small ones
    b = eng.batch(G, [Qs[i] for i in solved], want_hash=True, root_ranges=[ranges[i] for i in solved],
                  time_cap_s=120)
    rh = b.run()
    b.free()
    checked = 0
    for j, i in enumerate(solved):
        q = qs[i]
        try:
            ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(0, ranges[i][0], ranges[i][1]),
                          max_steps=2 * 10 ** 7)
        except O.OracleError:
            continue
        assert (int(rh["counts"][j]), int(rh["hashes"][j])) == (ref["count"], ref["hash"]), q.name
        checked += 1
    assert checked >= 4


def test_batch_root_chunks_on_a_wide_graph_against_closed_forms(eng):
    """Full root ranges wider than 2^20 vertices start from root chunks
    instead of a breadth-first pool: stars, the single edge and the single
    vertex against their closed forms on R-MAT scale 21."""
    g = gg.rmat_graph(21, 8, seed=21)
    assert g.n > (1 << 20)
    G = eng.load_graph(g.rowptr, g.col)
    d = np.diff(g.rowptr).astype(object)
    qs = [gg.Query(1, np.zeros((0, 2), np.int32)), gg.Query(2, [[0, 1]]), gg.pattern("S2"), gg.pattern("S3")]
    want = [g.n, int(sum(d)), int(sum(x * (x - 1) for x in d)), int(sum(x * (x - 1) * (x - 2) for x in d))]
    Qs = [eng.query(q.k, q.edges) for q in qs]
    for kw in [dict(), dict(chunk_words=1, warps_per_block=4)]:
        r = eng.count_batch(G, Qs, time_cap_s=120, **kw)
        assert [int(x) for x in r["counts"]] == want, kw
    # every embedding visited (no symmetry breaking, no arithmetic last level):
    # the stars of three leaves (7.5e14 embeddings here) are left out
    r = eng.count_batch(G, Qs[:3], time_cap_s=120, sym_break=0, arith_last=0)
    assert [int(x) for x in r["counts"]] == want[:3]
    G.free()


def test_per_query_work_is_exact_and_the_capped_selection_repeatable(eng, labelled):
    """A finished query's work (sgm_batch_query_work) does not depend on the
    scheduling: two runs, and runs in other launch shapes, report the same
    work for every query that finished, so the rule "finished within the cap"
    picks the same queries every time."""
    g = labelled
    G = eng.load_graph(g.rowptr, g.col, g.labels, 8)
    qs = _walk_queries(g, 96, 9, kmin=4, kmax=16)
    ranges = [(int(q.source[0]), int(q.source[0]) + 1) for q in qs]
    Qs = [eng.query(q.k, q.edges, q.labels) for q in qs]
    for Q in Qs:
        Q.order_greedy(G, root=0)
    cap = 1 << 20
    runs = []
    for kw in [dict(), dict(), dict(warps_per_block=4, split_min=64)]:
        b = eng.batch(G, Qs, root_ranges=ranges, work_cap=cap, time_cap_s=120, **kw)
        r = b.run(check=False)
        b.free()
        runs.append(r)
    keep = [{i for i in range(len(qs)) if r["statuses"][i] == 0 and int(r["work"][i]) <= cap} for r in runs]
    assert keep[0] == keep[1] == keep[2] and 0 < len(keep[0]) < len(qs)
    for i in keep[0]:
        assert int(runs[0]["work"][i]) == int(runs[1]["work"][i]) == int(runs[2]["work"][i]), qs[i].name
        assert int(runs[0]["counts"][i]) == int(runs[2]["counts"][i])
