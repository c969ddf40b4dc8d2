"""Parity of the CUDA engine (through its C ABI) with the CPU oracle:
bit-exact embedding counts, embedding hashes, listed embeddings, candidate
bitmaps and per-level partial-match counts, on seeded synthetic inputs that
span many warps, several BFS levels and ragged tails; plus edge cases and
the error codes of the boundary."""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine

    class CappedEngine(Engine):
        """Every run carries a search time cap, so that a case larger than
        expected ends with SGM_E_TIME_CAP instead of holding the GPU."""

        def count(self, *a, **kw):
            kw.setdefault("time_cap_s", 120.0)
            return super().count(*a, **kw)

        def enumerate(self, *a, **kw):
            kw.setdefault("time_cap_s", 120.0)
            return super().enumerate(*a, **kw)

    e = CappedEngine(0)
    yield e
    import gc
    gc.collect()


def _load(eng, g):
    return eng.load_graph(g.rowptr, g.col, g.labels, g.num_labels if g.labels is not None else 1)


def _q(eng, q):
    return eng.query(q.k, q.edges, q.labels)


def _sorted(rows):
    rows = np.asarray(rows)
    return rows[np.lexsort(rows.T[::-1])] if len(rows) else rows


def _random_connected_query(rng, k, extra, num_labels):
    edges = set()
    for v in range(1, k):
        edges.add((int(rng.integers(0, v)), v))
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
    rng.shuffle(pairs)
    for p in pairs[:extra]:
        edges.add(p)
    perm = rng.permutation(k)
    e = np.array([(perm[a], perm[b]) for a, b in sorted(edges)], dtype=np.int32)
    labels = rng.integers(0, num_labels, size=k).astype(np.int32) if num_labels > 1 else None
    return gg.Query(k, e, labels)


# ---------------------------------------------------------------------------
# the tiny labelled configuration: ER(2000, 0.004), 4 labels, tailed triangle
# ---------------------------------------------------------------------------
def test_er2000_tailed_triangle_full_parity(eng):
    g = gg.er_graph(2000, 0.004, 1, num_labels=4)
    q = gg.pattern("tailed_triangle")
    ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, want_rows=True)
    G, Q = _load(eng, g), _q(eng, q)
    r = eng.enumerate(G, Q, cap=4096)
    assert r["total"] == ref["count"] and r["hash"] == ref["hash"] and not r["truncated"]
    assert np.array_equal(_sorted(r["rows"].cpu().numpy()), ref["rows"])
    c = eng.count(G, Q, want_hash=True)
    assert (c["count"], c["hash"]) == (ref["count"], ref["hash"])
    assert eng.count(G, Q)["count"] == ref["count"]


# ---------------------------------------------------------------------------
# random small graphs and queries (labels 1..3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
def test_random_small_parity(eng, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 400))
    nl = int(rng.integers(1, 4))
    g = gg.er_graph(n, float(rng.uniform(0.02, 0.2)), seed, num_labels=nl)
    G = _load(eng, g)
    for _ in range(5):
        k = int(rng.integers(2, 7))
        q = _random_connected_query(rng, k, int(rng.integers(0, 4)), nl)
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, want_rows=True, cap=1 << 16)
        Q = _q(eng, q)
        r = eng.count(G, Q, want_hash=True)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), q.edges.tolist()
        assert eng.count(G, Q)["count"] == ref["count"]
        if ref["count"] <= 1 << 16:
            e = eng.enumerate(G, Q, cap=1 << 16)
            assert np.array_equal(_sorted(e["rows"].cpu().numpy()), ref["rows"])
        Q.free()
    G.free()


# ---------------------------------------------------------------------------
# unlabelled power-law graphs: the small patterns, count and hash modes,
# several initial-pool depths, work queue on and off
# ---------------------------------------------------------------------------
PATTERNS = ["K3", "K4", "K5", "C4", "C5", "P3", "P4", "P5", "S3", "house5d", "house6d"]


@pytest.fixture(scope="module")
def rmat10():
    # R-MAT scale 10, edge factor 2: hubs and skew, yet every pattern's full
    # embedding set stays small enough for the oracle (house6d ~1.4e7)
    return gg.rmat_graph(10, 2, seed=11)


@pytest.mark.parametrize("name", PATTERNS)
def test_rmat_patterns_parity(eng, rmat10, name):
    g = rmat10
    q = gg.pattern(name)
    ref = O.match(g.rowptr, g.col, None, q.k, q.edges)
    G, Q = _load(eng, g), _q(eng, q)
    qrp, qcol = gg.csr_from_edges(q.k, q.edges)
    aut = O.match(qrp, qcol, None, q.k, q.edges)["count"]  # |Aut(Q)|
    for kw in [dict(), dict(tau=1), dict(tau=10 ** 9), dict(split_min=0), dict(split_min=4, warps_per_block=2),
               dict(use_filter=0), dict(arith_last=0), dict(warps_per_block=1, blocks_per_sm=1),
               dict(sym_break=0), dict(sym_break=0, tau=1, split_min=8), dict(pool_chunk=0),
               dict(pool_chunk=4, split_min=2), dict(pool_chunk=16, tau=1, sym_break=0),
               dict(split_depth=32, split_min=4)]:
        r = eng.count(G, Q, want_hash=True, **kw)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), kw
        assert r["stats"]["aut_size"] == (aut if kw.get("sym_break", 1) else 1)
        c = eng.count(G, Q, **kw)
        assert c["count"] == ref["count"], kw
    e = eng.enumerate(G, Q, cap=1 << 16)
    assert e["total"] == ref["count"] and e["hash"] == ref["hash"]
    G.free()


def test_level_counts_match_filtered_prefix_counts(eng):
    g = gg.rmat_graph(10, 8, seed=12)
    g.labels = gg.labels_zipf(g.n, 3, 1.0, 12)
    g.num_labels = 3
    G = _load(eng, g)
    rng = np.random.default_rng(7)
    for _ in range(6):
        q = _random_connected_query(rng, int(rng.integers(3, 7)), int(rng.integers(0, 3)), 3)
        Q = _q(eng, q)
        Q.order_greedy(G)
        order = Q.order()
        bits = O.filter_bits(g.rowptr, g.col, g.labels, 3, q.k, q.edges, q.labels)
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, order=order, cand_bits=bits,
                      level_counts=True)
        for tau in (1, 10 ** 9):
            r = eng.count(G, Q, tau=tau, arith_last=0, sym_break=0)
            assert r["count"] == ref["count"]
            assert np.array_equal(r["level_counts"].astype(np.uint64), ref["level_counts"]), (tau, order)
        Q.free()


def test_filter_bitmaps_bit_exact(eng):
    import torch
    g = gg.rmat_graph(12, 8, seed=13)
    g.labels = gg.labels_zipf(g.n, 16, 1.0, 13)
    g.num_labels = 16
    G = _load(eng, g)
    for s in range(4):
        q = gg.walk_query(g, 8 + 4 * s, s % 2 == 0, 2, 500 + s)
        Q = _q(eng, q)
        for use_filter in (True, False):
            got = eng.filter_bits(G, Q, use_filter).cpu().numpy().view(np.uint32)
            if use_filter:
                ref = O.filter_bits(g.rowptr, g.col, g.labels, 16, q.k, q.edges, q.labels)
            else:
                ref = np.zeros_like(got)
                for u in range(q.k):
                    for v in np.nonzero(g.labels == q.labels[u])[0]:
                        ref[u, v >> 5] |= np.uint32(1 << (v & 31))
            assert np.array_equal(got, ref)
        Q.free()
    del torch


def test_order_independence_on_gpu(eng, rmat10):
    g = rmat10
    G = _load(eng, g)
    for name in ["house5d", "C5", "P5"]:
        q = gg.pattern(name)
        Q = _q(eng, q)
        ref = O.match(g.rowptr, g.col, None, q.k, q.edges)
        orders = [list(p) for p in itertools.permutations(range(q.k))
                  if all(any(((p[i], p[j]) in set(map(tuple, q.edges.tolist())) or
                              (p[j], p[i]) in set(map(tuple, q.edges.tolist()))) for j in range(i))
                         for i in range(1, q.k))]
        for order in orders[::7]:
            Q.set_order(order)
            r = eng.count(G, Q, want_hash=True)
            assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), order
            assert eng.count(G, Q)["count"] == ref["count"], order
        Q.free()


def test_root_slices_parity_and_additivity(eng, rmat10):
    g = rmat10
    G = _load(eng, g)
    for name in ["K4", "house6d", "C4"]:
        q = gg.pattern(name)
        Q = _q(eng, q)
        Q.order_greedy(G)
        root = int(Q.order()[0])
        cuts = [0, 1, 7, 100, 500, 501, 800, g.n]
        tot, h = 0, 0
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            r = eng.count(G, Q, want_hash=True, root_range=(lo, hi))
            ref = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(root, lo, hi))
            assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), (name, lo, hi)
            assert eng.count(G, Q, root_range=(lo, hi))["count"] == ref["count"]
            tot += r["count"]
            h = (h + r["hash"]) % (1 << 64)
        full = eng.count(G, Q, want_hash=True)
        assert (tot, h) == (full["count"], full["hash"])
        Q.free()


def test_labelled_walk_queries_parity(eng):
    # large random-walk queries on a uniformly labelled graph (Sec. 6.1's
    # large-query workload shape); where the full embedding set is beyond
    # the oracle's step budget, the slice rooted at the walk's seed vertex
    g = gg.rmat_graph(12, 8, seed=15)
    g.labels = gg.labels_uniform(g.n, 32, 15)
    g.num_labels = 32
    G = _load(eng, g)
    qs = gg.walk_query_set(g, [8, 8, 12, 12, 16, 16, 24, 32], [True, False] * 3 + [True, True], seed=15)
    checked = 0
    for q in qs:
        Q = _q(eng, q)
        try:
            ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, max_steps=2 * 10 ** 7)
            rng = None
        except O.OracleError:
            v = int(q.source[0])
            ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, root=(0, v, v + 1),
                          max_steps=2 * 10 ** 7)
            Q.order_greedy(G, root=0)
            rng = (v, v + 1)
        r = eng.count(G, Q, want_hash=True, root_range=rng)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), q.name
        assert eng.count(G, Q, root_range=rng)["count"] == ref["count"]
        checked += 1
        Q.free()
    assert checked == len(qs)


def test_enumerate_truncation(eng, rmat10):
    g = rmat10
    q = gg.pattern("P3")
    ref = O.match(g.rowptr, g.col, None, q.k, q.edges, want_rows=True, cap=1 << 22)
    G, Q = _load(eng, g), _q(eng, q)
    cap = ref["count"] // 3
    r = eng.enumerate(G, Q, cap=cap)
    assert r["truncated"] and r["written"] == cap and r["total"] == ref["count"] and r["hash"] == ref["hash"]
    rows = r["rows"].cpu().numpy()
    assert len(np.unique(rows, axis=0)) == cap
    full = {tuple(x) for x in ref["rows"].tolist()}
    assert all(tuple(x) in full for x in rows.tolist())


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_edge_cases(eng):
    # graph with isolated vertices only
    rp, col = np.zeros(6, np.int64), np.zeros(0, np.int32)
    G = eng.load_graph(rp, col)
    for name in ["K3", "P3"]:
        q = gg.pattern(name)
        assert eng.count(G, _q(eng, q))["count"] == 0
    # single-vertex query counts vertices with the label
    g = gg.er_graph(300, 0.02, 3, num_labels=3)
    G = _load(eng, g)
    Q1 = eng.query(1, np.zeros((0, 2), np.int32), [2])
    assert eng.count(G, Q1)["count"] == int((g.labels == 2).sum())
    r = eng.count(G, Q1, want_hash=True)
    ref = O.match(g.rowptr, g.col, g.labels, 1, np.zeros((0, 2), np.int32), [2])
    assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])
    # two-vertex query = directed edges with those labels
    Q2 = eng.query(2, [[0, 1]], [0, 1])
    ref = O.match(g.rowptr, g.col, g.labels, 2, [[0, 1]], [0, 1])
    assert eng.count(G, Q2)["count"] == ref["count"]
    assert eng.count(G, Q2, want_hash=True)["hash"] == ref["hash"]
    # query larger than the graph
    tiny = gg.er_graph(5, 1.0, 1)
    Gt = _load(eng, tiny)
    assert eng.count(Gt, _q(eng, gg.pattern("K5")))["count"] == 120
    assert eng.count(Gt, _q(eng, gg.pattern("P6")))["count"] == 0
    # empty root range
    Qk = _q(eng, gg.pattern("K3"))
    assert eng.count(G, Qk, root_range=(50, 50))["count"] == 0
    # a 32-vertex path inside a 40-cycle
    c = gg.pattern("C40")
    rp, col = gg.csr_from_edges(40, c.edges)
    Gc = eng.load_graph(rp, col)
    p = gg.pattern("P32")
    assert eng.count(Gc, _q(eng, p), want_hash=True)["count"] == 80
    assert eng.count(Gc, _q(eng, p))["count"] == 80


def test_error_codes(eng):
    from paper_2604_10601_gb300 import sgm
    def code(fn):
        with pytest.raises(sgm.SgmError) as ei:
            fn()
        return ei.value.status
    # unsorted row / self loop / asymmetric / out of range
    rp = np.array([0, 2, 3, 4], np.int64)
    assert code(lambda: eng.load_graph(rp, np.array([2, 1, 0, 0], np.int32))) == sgm.SGM_E_GRAPH_UNSORTED
    assert code(lambda: eng.load_graph(np.array([0, 1, 1], np.int64), np.array([0], np.int32))) == \
        sgm.SGM_E_GRAPH_SELF_LOOP
    assert code(lambda: eng.load_graph(np.array([0, 1, 1], np.int64), np.array([1], np.int32))) == \
        sgm.SGM_E_GRAPH_ASYMMETRIC
    assert code(lambda: eng.load_graph(np.array([0, 1, 2], np.int64), np.array([1, 5], np.int32))) == \
        sgm.SGM_E_GRAPH_RANGE
    assert code(lambda: eng.load_graph(np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32))) == \
        sgm.SGM_E_GRAPH_RANGE
    g = gg.er_graph(50, 0.1, 1, num_labels=2)
    assert code(lambda: eng.load_graph(g.rowptr, g.col, np.full(50, 7, np.int32), 2)) == sgm.SGM_E_LABEL_RANGE
    G = _load(eng, g)
    assert code(lambda: eng.query(3, [[0, 1]])) == sgm.SGM_E_QUERY_DISCONNECTED
    assert code(lambda: eng.query(33, [[i, i + 1] for i in range(32)])) == sgm.SGM_E_QUERY_TOO_LARGE
    assert code(lambda: eng.query(2, [[0, 0]])) == sgm.SGM_E_QUERY_INVALID
    assert code(lambda: eng.query(2, [[0, 1], [1, 0]])) == sgm.SGM_E_QUERY_INVALID
    Q = eng.query(3, [[0, 1], [1, 2]])
    assert code(lambda: Q.set_order([0, 2, 1])) == sgm.SGM_E_ORDER_NOT_CONNECTED
    Ql = eng.query(2, [[0, 1]], [0, 5])
    assert code(lambda: eng.count(G, Ql)) == sgm.SGM_E_LABEL_RANGE
    # the engine stays usable after every error
    assert eng.count(G, Q)["count"] == O.match(g.rowptr, g.col, g.labels, 3, [[0, 1], [1, 2]])["count"]


def test_time_cap_returns_unsolved(eng):
    from paper_2604_10601_gb300 import sgm
    g = gg.rmat_graph(16, 16, seed=16)
    G, Q = _load(eng, g), _q(eng, gg.pattern("P5"))
    with pytest.raises(sgm.SgmError) as ei:
        eng.count(G, Q, want_hash=True, time_cap_s=0.002)
    assert ei.value.status == sgm.SGM_E_TIME_CAP
    assert eng.count(G, _q(eng, gg.pattern("S2")))["count"] == int((g.degrees() * (g.degrees() - 1)).sum())


# ---------------------------------------------------------------------------
# RMAT scale 20, edge factor 16 (the unlabelled power-law workload): closed
# forms over the whole graph, oracle parity on seeded root slices
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def rmat20():
    return gg.rmat_graph(20, 16, seed=1)


def test_rmat20_closed_forms(eng, rmat20):
    # stars with 1 and 2 leaves over the whole graph (sum_v d!/(d-k)!); the
    # 3-leaf star visits ~3.5e10 wedges here, so it is checked at scale 16
    import math
    for g, leaves_set in ((rmat20, (1, 2)), (gg.rmat_graph(16, 16, seed=2), (3,))):
        G = _load(eng, g)
        for leaves in leaves_set:
            expect = sum(math.perm(int(x), leaves) for x in g.degrees() if x >= leaves)
            r = eng.count(G, _q(eng, gg.pattern(f"S{leaves}")), time_cap_s=60)
            assert r["count"] == expect, leaves
        G.free()


def _slice_roots(g):
    """Seeded single-vertex root slices whose embedding sets the oracle lists
    in well under a second: low-degree roots whose neighbours have a small
    degree sum, mid-degree ones, and high-degree ones for the cliques."""
    deg = g.degrees().astype(np.int64)
    src = np.repeat(np.arange(g.n), deg)
    s1 = np.bincount(src, weights=deg[g.col], minlength=g.n)
    classes = {}
    for cls, (dlo, dhi, smax, seed, cnt) in {"low": (2, 6, 4000, 20, 2), "mid": (10, 30, 60000, 21, 2),
                                              "high": (60, 120, 300000, 22, 2)}.items():
        ok = np.nonzero((deg >= dlo) & (deg <= dhi) & (s1 <= smax))[0]
        classes[cls] = [int(v) for v in np.random.default_rng(seed).choice(ok, size=cnt, replace=False)]
    return classes


SLICE_PLAN = {"K4": (0, ("low", "mid", "high")), "K5": (0, ("mid", "high")), "C4": (0, ("low", "mid")),
              "P5": (2, ("low",)), "house5d": (0, ("mid", "high")), "house6d": (0, ("low", "mid"))}


@pytest.mark.parametrize("name", list(SLICE_PLAN))
def test_rmat20_root_slices(eng, rmat20, name):
    g = rmat20
    G = _load(eng, g)
    q = gg.pattern(name)
    Q = _q(eng, q)
    root, classes = SLICE_PLAN[name]
    Q.order_greedy(G, root=root)
    assert int(Q.order()[0]) == root
    roots = _slice_roots(g)
    for cls in classes:
        for v in roots[cls]:
            ref = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(root, v, v + 1), max_steps=3 * 10 ** 8)
            r = eng.count(G, Q, want_hash=True, root_range=(v, v + 1))
            assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), (name, v)
            assert eng.count(G, Q, root_range=(v, v + 1))["count"] == ref["count"]
    # a contiguous slice of the highest ids (isolated and degree-1 vertices)
    lo = g.n - 4096
    ref = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(root, lo, g.n), max_steps=3 * 10 ** 8)
    assert eng.count(G, Q, root_range=(lo, g.n))["count"] == ref["count"]
