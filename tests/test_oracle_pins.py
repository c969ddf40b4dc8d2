"""Pins for the CPU oracle against facts fixed outside the oracle itself:
published test vectors, brute force over all injective maps, closed-form
embedding counts, a hand-computed filter example, and invariants of
Definition 1 (order independence, slice additivity, automorphism
divisibility, monotonicity in query edges, walk-query self-embedding)."""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sorted_rows(r):
    r = np.asarray(r)
    return r[np.lexsort(r.T[::-1])] if len(r) else r


def _random_connected_query(rng, k, extra, num_labels):
    edges = set()
    for v in range(1, k):
        u = int(rng.integers(0, v))
        edges.add((u, v))
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
    rng.shuffle(pairs)
    for p in pairs[:extra]:
        edges.add(p)
    perm = rng.permutation(k)  # relabel so vertex 0 is not always the tree root
    e = np.array([(perm[a], perm[b]) for a, b in sorted(edges)], dtype=np.int32)
    labels = rng.integers(0, num_labels, size=k).astype(np.int32) if num_labels > 1 else None
    return gg.Query(k, e, labels)


# ---------------------------------------------------------------------------
# the hash mixer: published SplitMix64 outputs
# ---------------------------------------------------------------------------
def test_mix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for state, out in rows:
        assert O.mix64(int(state, 16)) == int(out, 16)


def test_hash_is_sum_over_listed_rows():
    g = gg.er_graph(11, 0.5, 7)
    q = gg.pattern("P4")
    r = O.match(g.rowptr, g.col, None, q.k, q.edges, want_rows=True)
    assert r["count"] == len(r["rows"]) > 0
    assert r["hash"] == sum(O.embedding_hash(row) for row in r["rows"]) % (1 << 64)
    # the per-row hash is indexed by query vertex: permuting values changes it
    row = r["rows"][0]
    assert O.embedding_hash(row) != O.embedding_hash(row[::-1])


# ---------------------------------------------------------------------------
# brute force (every injective map) on tiny graphs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(12))
def test_oracle_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 12))
    nl = int(rng.integers(1, 4))
    g = gg.er_graph(n, float(rng.uniform(0.3, 0.7)), seed, num_labels=max(nl, 1), label_seed=seed + 100)
    labels = g.labels if nl > 1 else None
    for _ in range(4):
        k = int(rng.integers(2, 7))
        q = _random_connected_query(rng, k, int(rng.integers(0, 3)), nl)
        a = O.match(g.rowptr, g.col, labels, q.k, q.edges, q.labels, want_rows=True)
        b = O.brute(g.rowptr, g.col, labels, q.k, q.edges, q.labels)
        assert a["count"] == b["count"]
        assert a["hash"] == b["hash"]
        assert np.array_equal(_sorted_rows(a["rows"]), _sorted_rows(b["rows"]))


def test_brute_force_counts_all_injections_on_complete_graph():
    # on K_n with the empty-edge query on k vertices every injective map counts
    rowptr, col = gg.csr_from_edges(6, [(i, j) for i in range(6) for j in range(i + 1, 6)])
    for k in range(1, 5):
        b = O.brute(rowptr, col, None, k, np.zeros((0, 2), np.int32))
        assert b["count"] == math.perm(6, k)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 7, 9])
def test_clique_in_clique(n):
    rowptr, col = gg.csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    for k in range(2, min(n, 6) + 1):
        q = gg.pattern(f"K{k}")
        assert O.match(rowptr, col, None, q.k, q.edges)["count"] == math.factorial(n) // math.factorial(n - k)


@pytest.mark.parametrize("n", [3, 4, 5, 8, 13])
def test_cycle_in_itself(n):
    q = gg.pattern(f"C{n}")
    rowptr, col = gg.csr_from_edges(n, q.edges)
    assert O.match(rowptr, col, None, q.k, q.edges)["count"] == 2 * n


@pytest.mark.parametrize("seed", [1, 2])
def test_star_formula(seed):
    g = gg.rmat_graph(9, 8, seed=seed)
    d = g.degrees()
    for leaves in (1, 2, 3):
        q = gg.pattern(f"S{leaves}")
        expect = sum(math.perm(int(x), leaves) for x in d if x >= leaves)
        assert O.match(g.rowptr, g.col, None, q.k, q.edges)["count"] == expect


def _triangles_degree_oriented(rowptr, col):
    """Triangles counted once each: orient every edge from lower to higher
    (degree, id) and intersect out-neighbourhoods (independent of the oracle)."""
    n = len(rowptr) - 1
    deg = np.diff(rowptr)
    key = lambda v: (deg[v], v)
    out = []
    for v in range(n):
        nb = col[rowptr[v]:rowptr[v + 1]]
        out.append(set(int(w) for w in nb if key(w) > key(v)))
    t = 0
    for v in range(n):
        for w in out[v]:
            t += len(out[v] & out[w])
    return t


def test_triangle_count_independent():
    g = gg.rmat_graph(10, 8, seed=3)
    q = gg.pattern("K3")
    assert O.match(g.rowptr, g.col, None, 3, q.edges)["count"] == 6 * _triangles_degree_oriented(g.rowptr, g.col)


def test_four_cycle_trace_formula():
    # closed 4-walks minus the degenerate ones: tr(A^4) - 2 sum d^2 + 2|E|
    g = gg.er_graph(60, 0.12, 5)
    n = g.n
    A = np.zeros((n, n), dtype=np.int64)
    for v in range(n):
        A[v, g.neighbors(v)] = 1
    d = A.sum(1)
    A2 = A @ A
    expect = int(np.trace(A2 @ A2) - 2 * (d * d).sum() + d.sum())
    q = gg.pattern("C4")
    assert O.match(g.rowptr, g.col, None, 4, q.edges)["count"] == expect


def test_tailed_triangle_closed_form_er2000():
    # triangle (a,b,c) with labels (0,1,2) plus a pendant w in N(a) with label 0
    g = gg.er_graph(2000, 0.004, 1, num_labels=4)
    q = gg.pattern("tailed_triangle")
    L = g.labels
    expect = 0
    for a in np.nonzero(L == 0)[0]:
        na = set(int(x) for x in g.neighbors(a))
        w0 = sum(1 for x in na if L[x] == 0)
        for b in na:
            if L[b] != 1:
                continue
            for c in g.neighbors(b):
                if L[c] == 2 and int(c) in na:
                    expect += w0
    r = O.match(g.rowptr, g.col, L, 4, q.edges, q.labels, want_rows=True)
    assert r["count"] == expect
    assert expect > 0


# ---------------------------------------------------------------------------
# the candidate filter: hand-computed example, soundness, unlabelled closed form
# ---------------------------------------------------------------------------
def _read_filter_golden():
    d = {"cand": {}}
    for line in open(os.path.join(GOLDEN, "filter_tiny.txt")):
        if not line.strip() or line[0] == "#":
            continue
        f = line.split()
        if f[0] == "cand":
            d["cand"][int(f[1])] = [int(x) for x in f[2:]]
        else:
            d[f[0]] = [int(x) for x in f[1:]]
    return d


def test_filter_hand_example():
    d = _read_filter_golden()
    n = d["n"][0]
    rowptr, col = gg.csr_from_edges(n, np.array(d["edges"]).reshape(-1, 2))
    bits = O.filter_bits(rowptr, col, d["labels"], 2, 3, d["qedges"], d["qlabels"])
    for u, cands in d["cand"].items():
        got = [v for v in range(n) if (bits[u, v >> 5] >> (v & 31)) & 1]
        assert got == cands
    r = O.match(rowptr, col, d["labels"], 3, d["qedges"], d["qlabels"])
    assert r["count"] == d["count"][0]


def test_filter_unlabelled_is_degree_threshold():
    g = gg.rmat_graph(9, 8, seed=4)
    q = gg.pattern("S3")
    bits = O.filter_bits(g.rowptr, g.col, None, 1, q.k, q.edges)
    deg = g.degrees()
    for u, need in [(0, 3), (1, 1), (2, 1), (3, 1)]:
        got = np.array([(bits[u, v >> 5] >> (v & 31)) & 1 for v in range(g.n)], dtype=bool)
        assert np.array_equal(got, deg >= need)


@pytest.mark.parametrize("seed", range(4))
def test_filter_sound_and_count_preserving(seed):
    rng = np.random.default_rng(seed)
    g = gg.er_graph(300, 0.03, seed, num_labels=3)
    q = _random_connected_query(rng, 5, 2, 3)
    bits = O.filter_bits(g.rowptr, g.col, g.labels, 3, q.k, q.edges, q.labels)
    full = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, want_rows=True)
    filt = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, cand_bits=bits)
    assert full["count"] == filt["count"] and full["hash"] == filt["hash"]
    for row in full["rows"]:
        for u, v in enumerate(row):
            assert (bits[u, v >> 5] >> (v & 31)) & 1


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def _connected_orders(q):
    adj = [set() for _ in range(q.k)]
    for a, b in q.edges:
        adj[a].add(int(b))
        adj[b].add(int(a))
    for perm in itertools.permutations(range(q.k)):
        if all(adj[perm[i]] & set(perm[:i]) for i in range(1, q.k)):
            yield list(perm)


@pytest.mark.parametrize("name", ["P4", "C4", "house5d", "K4", "S3"])
def test_order_independence_exhaustive(name):
    g = gg.rmat_graph(7, 4, seed=5)
    q = gg.pattern(name)
    ref = O.match(g.rowptr, g.col, None, q.k, q.edges)
    for order in _connected_orders(q):
        r = O.match(g.rowptr, g.col, None, q.k, q.edges, order=order)
        assert (r["count"], r["hash"]) == (ref["count"], ref["hash"])


def test_level_counts_are_prefix_embedding_counts():
    rng = np.random.default_rng(9)
    g = gg.er_graph(10, 0.5, 9, num_labels=2, label_seed=3)
    q = _random_connected_query(rng, 5, 2, 2)
    order = next(_connected_orders(q))
    r = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, order=order, level_counts=True)
    for i in range(q.k):
        keep = order[:i + 1]
        idx = {u: j for j, u in enumerate(keep)}
        sub = [(idx[a], idx[b]) for a, b in q.edges if a in idx and b in idx]
        sub = np.array(sub, dtype=np.int32).reshape(-1, 2)
        b = O.brute(g.rowptr, g.col, g.labels, i + 1, sub, q.labels[keep])
        assert int(r["level_counts"][i]) == b["count"]
    assert int(r["level_counts"][-1]) == r["count"]


def test_root_slice_additivity():
    g = gg.rmat_graph(8, 4, seed=6)
    q = gg.pattern("house5d")
    full = O.match(g.rowptr, g.col, None, q.k, q.edges)
    for root_u in (0, 4):
        cuts = [0, 10, 11, 33, 90, g.n]
        tot, h = 0, 0
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            r = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(root_u, lo, hi))
            tot += r["count"]
            h = (h + r["hash"]) % (1 << 64)
        assert (tot, h) == (full["count"], full["hash"])


@pytest.mark.parametrize("name", ["K4", "C4", "C5", "house5d", "house6d", "S3", "P5"])
def test_count_divisible_by_automorphisms(name):
    g = gg.rmat_graph(7, 4, seed=7)
    q = gg.pattern(name)
    qrp, qcol = gg.csr_from_edges(q.k, q.edges)
    aut = O.match(qrp, qcol, None, q.k, q.edges)["count"]  # |Aut(Q)|: Q embedded in itself
    expect_aut = {"K4": 24, "C4": 8, "C5": 10, "house5d": 2, "house6d": 1, "S3": 6, "P5": 2}[name]
    assert aut == expect_aut
    c = O.match(g.rowptr, g.col, None, q.k, q.edges)["count"]
    assert c % aut == 0


def test_adding_edge_never_increases_count():
    g = gg.er_graph(80, 0.1, 8)
    rng = np.random.default_rng(3)
    for _ in range(5):
        q = _random_connected_query(rng, 5, 0, 1)
        base = O.match(g.rowptr, g.col, None, q.k, q.edges)["count"]
        present = set(map(tuple, np.sort(q.edges, axis=1).tolist()))
        missing = [(i, j) for i in range(5) for j in range(i + 1, 5) if (i, j) not in present]
        e = missing[int(rng.integers(0, len(missing)))]
        more = O.match(g.rowptr, g.col, None, q.k, np.vstack([q.edges, [e]]))["count"]
        assert more <= base


@pytest.mark.parametrize("dense", [True, False])
def test_walk_query_contains_its_source(dense):
    g = gg.rmat_graph(10, 8, seed=9)
    g.labels = gg.labels_zipf(g.n, 4, 1.0, 9)
    g.num_labels = 4
    for s in range(3):
        q = gg.walk_query(g, 6, dense, 1, 1000 + s)
        # the slice M[0] = source[0] keeps the listing small
        r = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels, want_rows=True,
                    root=(0, int(q.source[0]), int(q.source[0]) + 1))
        assert not r.get("truncated")
        assert any(np.array_equal(row, q.source) for row in r["rows"])


def test_closed_form_helpers_against_reference_counts():
    # the C helpers that pin full-size GPU counts, pinned themselves: the
    # Python degree-oriented triangle count, scipy's tr(A^4), and the oracle
    import scipy.sparse as sp
    import closed_forms as CF
    for seed in (3, 4):
        g = gg.rmat_graph(10, 8, seed=seed)
        assert CF.triangles(g.rowptr, g.col) == _triangles_degree_oriented(g.rowptr, g.col)
        A = sp.csr_matrix((np.ones(len(g.col), np.int64), g.col, g.rowptr), shape=(g.n, g.n))
        A2 = A @ A
        assert CF.trace_a4(g.rowptr, g.col) == int(A2.multiply(A2).sum())
        q = gg.pattern("C4")
        assert CF.c4_embeddings(g.rowptr, g.col) == O.match(g.rowptr, g.col, None, 4, q.edges)["count"]
