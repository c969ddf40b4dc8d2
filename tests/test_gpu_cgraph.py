"""The candidate graph G' on the GPU (sgm_cgraph_build, App. C) against the
candidate-graph oracle: for every query edge in both directions, the
vertices of C(u) and the lists N(v) ∩ C(u2) bit-exact, with the filter's
sets and with refined ones (several round counts), on graphs whose bitmaps
end in ragged words; searches on G' (sgm_count_cgraph) give the oracle's
counts and hashes, and per-level counts equal to the oracle's search over
the same candidate sets; the edge cases and errors of the boundary."""
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


def _cases():
    out = []
    for s in range(5):
        rng = np.random.default_rng(170 + s)
        n = [1000, 2007, 1500, 777, 3001][s]
        L = [2, 3, 4, 3, 5][s]
        g = gg.er_graph(n, 8.0 / n, 1900 + s, num_labels=L)
        k = int(rng.integers(3, 9))
        edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}
        pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
        rng.shuffle(pairs)
        edges |= set(pairs[:int(rng.integers(0, 3))])
        q = gg.Query(k, np.array(sorted(edges), dtype=np.int32), rng.integers(0, L, size=k).astype(np.int32))
        out.append((g, L, q))
    g = gg.rmat_graph(11, 8, 0.57, 0.19, 0.19, seed=7)
    g.labels = gg.labels_zipf(g.n, 6, 1.0, 8)
    g.num_labels = 6
    out.append((g, 6, gg.walk_query(g, 6, True, 1, 60)))
    # (listed last among the labelled cases: its lists are compared, its
    # count is beyond the oracle's reach)
    out.append((g, 6, gg.walk_query(g, 8, False, 1, 61)))
    gu = gg.rmat_graph(9, 4, 0.57, 0.19, 0.19, seed=9)
    out.append((gu, 1, gg.pattern("house5d")))
    return out


CASES = _cases()
SEARCHABLE = [0, 1, 2, 3, 4, 5, 7]  # the cases the oracle counts in seconds


def _load(eng, g, L):
    if g.labels is None:
        return eng.load_graph(g.rowptr, g.col)
    return eng.load_graph(g.rowptr, g.col, g.labels, L)


def _oracle_sets(g, L, q, rounds):
    c0 = CG.bits_to_sets(O.filter_bits(g.rowptr, g.col, g.labels, L, q.k, q.edges, q.labels), g.n)
    if rounds == 0:
        return c0
    return CG.refine(g.rowptr, g.col, q.k, q.edges, c0, max_rounds=rounds)[0]


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_candidate_edges_match_the_oracle(eng, ci):
    g, L, q = CASES[ci]
    G = _load(eng, g, L)
    Q = eng.query(q.k, q.edges, q.labels)
    for rounds in (0, 1, 64):
        want = CG.candidate_edges(g.rowptr, g.col, q.k, q.edges, _oracle_sets(g, L, q, rounds))
        C = eng.candidate_graph(G, Q, refine_rounds=rounds)
        assert len(want) == 2 * len(q.edges)
        for (u, u2), (vs, ptr, adj) in want.items():
            gvs, gptr, gadj = C.edge(u, u2)
            assert np.array_equal(gvs, vs), (ci, rounds, u, u2)
            assert np.array_equal(gptr, ptr), (ci, rounds, u, u2)
            assert np.array_equal(gadj, adj), (ci, rounds, u, u2)
        C.free()
    Q.free()
    G.free()


@pytest.mark.parametrize("ci", SEARCHABLE)
def test_search_on_the_candidate_graph(eng, ci):
    g, L, q = CASES[ci]
    G = _load(eng, g, L)
    Q = eng.query(q.k, q.edges, q.labels)
    Q.order_greedy(G)
    full = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, max_steps=1 << 30)
    for rounds in (0, 64):
        C = eng.candidate_graph(G, Q, refine_rounds=rounds)
        r = C.count(want_hash=True, time_cap_s=CAP)
        assert (r["count"], r["hash"]) == (full["count"], full["hash"]), (ci, rounds)
        assert C.count(time_cap_s=CAP)["count"] == full["count"]
        # per-level counts are those of a search over the same sets
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, order=Q.order(),
                      cand_bits=CG.sets_to_bits(_oracle_sets(g, L, q, rounds)), level_counts=True,
                      max_steps=1 << 30)
        for kw in (dict(tau=1), dict(tau=64), dict(tau=10 ** 6, split_min=2)):
            r = C.count(arith_last=0, sym_break=0, time_cap_s=CAP, **kw)
            assert np.array_equal(r["level_counts"].astype(np.uint64), ref["level_counts"]), (ci, rounds, kw)
        # and the plain search over the same refined sets agrees
        assert eng.count(G, Q, refine_rounds=rounds, time_cap_s=CAP)["count"] == full["count"]
        C.free()
    Q.free()
    G.free()


def test_candidate_graph_edge_cases_and_errors(eng):
    from paper_2604_10601_gb300 import sgm
    g = gg.er_graph(300, 0.02, 3, num_labels=2)
    G = eng.load_graph(g.rowptr, g.col, g.labels, 2)
    # a single-vertex query: no edges, the search counts C(u)
    Q1 = eng.query(1, np.zeros((0, 2), dtype=np.int32), np.array([1], dtype=np.int32))
    C1 = eng.candidate_graph(G, Q1)
    assert C1.count()["count"] == int((g.labels == 1).sum())
    with pytest.raises(sgm.SgmError) as ei:
        C1.edge(0, 0)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    C1.free()
    # a label no vertex carries: empty sets and lists
    Q = eng.query(3, np.array([[0, 1], [1, 2]], dtype=np.int32), np.array([0, 1, 0], dtype=np.int32))
    Qe = eng.query(2, np.array([[0, 1]], dtype=np.int32), np.array([0, 1], dtype=np.int32))
    g2 = gg.Graph(g.rowptr, g.col, np.zeros(g.n, dtype=np.int32), 2)
    G2 = eng.load_graph(g2.rowptr, g2.col, g2.labels, 2)
    Ce = eng.candidate_graph(G2, Qe, use_filter=False)  # (the label test alone: C(0) is every vertex)
    vs, ptr, adj = Ce.edge(1, 0)
    assert len(vs) == 0 and np.array_equal(ptr, [0]) and len(adj) == 0
    vs, ptr, adj = Ce.edge(0, 1)
    assert len(vs) > 0 and ptr[-1] == 0 and len(adj) == 0
    assert Ce.count()["count"] == 0
    Ce.free()
    # the object belongs to one graph and one query
    C = eng.candidate_graph(G, Q)
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_count_cgraph(eng.handle, G2.handle, Q.handle, C.handle, eng.opts())
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    with pytest.raises(sgm.SgmError) as ei:
        C.count(exec_model=2)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    with pytest.raises(sgm.SgmError) as ei:
        eng.candidate_graph(G, Q, refine_rounds=-1)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    ref = O.match(g.rowptr, g.col, g.labels, 3, [[0, 1], [1, 2]], [0, 1, 0])
    assert C.count()["count"] == ref["count"]
    C.free()
    G2.free()
    G.free()
