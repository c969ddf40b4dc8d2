"""The candidate-set refinement on the GPU (sgm_refine, opts.refine_rounds)
against the candidate-graph oracle: refined bitmaps and round counts
bit-exact for every number of rounds, on graphs with ragged bitmap tails;
counts, hashes, listings and per-level partial-match counts of refined runs
equal to the oracle's search over the same refined sets; and the error
cases of the boundary."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from oracle import candidate_graph as CG

pytestmark = pytest.mark.gpu

CAP = 120.0


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine
    e = Engine(0)
    yield e
    import gc
    gc.collect()


def _labelled_cases():
    out = []
    for s in range(6):
        rng = np.random.default_rng(70 + s)
        n = [1000, 2007, 1500, 777, 3000, 2048][s]
        L = [2, 3, 4, 3, 5, 2][s]
        g = gg.er_graph(n, 8.0 / n, 900 + s, num_labels=L)
        k = int(rng.integers(3, 9))
        edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}
        pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
        rng.shuffle(pairs)
        edges |= set(pairs[:int(rng.integers(0, 3))])
        q = gg.Query(k, np.array(sorted(edges), dtype=np.int32), rng.integers(0, L, size=k).astype(np.int32))
        out.append((g, L, q))
    g = gg.rmat_graph(12, 8, 0.57, 0.19, 0.19, seed=5)
    g.labels = gg.labels_zipf(g.n, 8, 1.0, 6)
    g.num_labels = 8
    for s in range(3):
        out.append((g, 8, gg.walk_query(g, 6 + 3 * s, s % 2 == 0, 2, 40 + s)))
    return out


def _oracle_refined(g, L, q, max_rounds=None):
    c0 = CG.bits_to_sets(O.filter_bits(g.rowptr, g.col, g.labels, L, q.k, q.edges, q.labels), g.n)
    return CG.refine(g.rowptr, g.col, q.k, q.edges, c0, max_rounds=max_rounds)


def test_refined_bitmaps_match_the_oracle(eng):
    for g, L, q in _labelled_cases():
        G = eng.load_graph(g.rowptr, g.col, g.labels, L)
        Q = eng.query(q.k, q.edges, q.labels)
        for max_rounds in (0, 1, 2, 64):
            got, rounds = eng.refine_bits(G, Q, max_rounds)
            got = got.cpu().numpy().view(np.uint32)
            want, want_rounds = _oracle_refined(g, L, q, max_rounds)
            assert rounds == want_rounds, (g.n, q.k, max_rounds)
            assert np.array_equal(got, CG.sets_to_bits(want)), (g.n, q.k, max_rounds)
        Q.free()
        G.free()


def test_refined_runs_count_exactly(eng):
    # the larger walk queries of the R-MAT graph have 1e8 and more embeddings
    # even from one root: their bitmaps are compared above, their counts not
    for g, L, q in _labelled_cases()[:7]:
        G = eng.load_graph(g.rowptr, g.col, g.labels, L)
        Q = eng.query(q.k, q.edges, q.labels)
        Q.order_greedy(G)
        order = Q.order()
        refined, _ = _oracle_refined(g, L, q)
        full = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels)
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, order=order,
                      cand_bits=CG.sets_to_bits(refined), level_counts=True)
        assert (ref["count"], ref["hash"]) == (full["count"], full["hash"])
        r = eng.count(G, Q, want_hash=True, refine_rounds=64, time_cap_s=CAP)
        assert (r["count"], r["hash"]) == (full["count"], full["hash"])
        # the search ran over the refined sets: its per-level counts are the
        # oracle's over the same sets
        r = eng.count(G, Q, refine_rounds=64, arith_last=0, sym_break=0, tau=1, time_cap_s=CAP)
        assert np.array_equal(r["level_counts"].astype(np.uint64), ref["level_counts"])
        assert eng.count(G, Q, refine_rounds=2, time_cap_s=CAP)["count"] == full["count"]
        Q.free()
        G.free()


def test_refined_listing_and_root_slices(eng):
    g, L, q = _labelled_cases()[1]
    G = eng.load_graph(g.rowptr, g.col, g.labels, L)
    Q = eng.query(q.k, q.edges, q.labels)
    Q.order_greedy(G)
    full = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, want_rows=True)
    e = eng.enumerate(G, Q, max(full["count"], 1), refine_rounds=64, time_cap_s=CAP)
    rows = e["rows"].cpu().numpy()
    rows = rows[np.lexsort(rows.T[::-1])] if len(rows) else rows
    assert e["total"] == full["count"] and np.array_equal(rows, full["rows"])
    root = int(Q.order()[0])
    cuts = [0, g.n // 3, g.n // 2 + 5, g.n]
    tot = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        r = eng.count(G, Q, root_range=(a, b), refine_rounds=64, time_cap_s=CAP)
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(root, a, b))
        assert r["count"] == ref["count"]
        tot += r["count"]
    assert tot == full["count"]
    Q.free()
    G.free()


def test_refinement_edge_cases_and_errors(eng):
    from paper_2604_10601_gb300 import sgm
    g = gg.er_graph(300, 0.02, 3, num_labels=2)
    G = eng.load_graph(g.rowptr, g.col, g.labels, 2)
    Q1 = eng.query(1, np.zeros((0, 2), dtype=np.int32), np.array([1], dtype=np.int32))
    got, rounds = eng.refine_bits(G, Q1, 8)  # no query edges: nothing to refine
    assert rounds == 0
    assert np.array_equal(got.cpu().numpy().view(np.uint32),
                          O.filter_bits(g.rowptr, g.col, g.labels, 2, 1, np.zeros((0, 2), np.int32), [1]))
    assert eng.count(G, Q1, refine_rounds=8)["count"] == int((g.labels == 1).sum())
    Q = eng.query(3, np.array([[0, 1], [1, 2]], dtype=np.int32), np.array([0, 1, 0], dtype=np.int32))
    with pytest.raises(sgm.SgmError) as ei:
        eng.refine_bits(G, Q, -1)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    with pytest.raises(sgm.SgmError) as ei:
        eng.count(G, Q, refine_rounds=-2)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    with pytest.raises(sgm.SgmError) as ei:
        eng.count_batch(G, [Q], refine_rounds=1)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    with pytest.raises(TypeError):
        eng.count(G, Q, refine_round=1)  # misspelt option
    # the engine is still usable after the rejected calls
    ref = O.match(g.rowptr, g.col, g.labels, 3, [[0, 1], [1, 2]], [0, 1, 0])
    assert eng.count(G, Q, refine_rounds=3)["count"] == ref["count"]
    Q.free()
    Q1.free()
    G.free()
