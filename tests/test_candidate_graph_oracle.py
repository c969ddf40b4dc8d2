"""Pins for the candidate-graph oracle (oracle/candidate_graph.py), against
facts fixed outside it: a hand-worked cascade (tests/golden), brute force
over all embeddings (every embedding lies in G'), exact counts and hashes
when the search is restricted to the refined sets, the support condition
at the fixed point, the same fixed point from in-place updates in another
order (the greatest fixed point is unique), and, for tree queries with
label-only starting sets, the classical fact that the refined sets are
exactly the images of label-preserving homomorphisms."""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from oracle import candidate_graph as CG

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    d = {"edge": []}
    for line in open(os.path.join(GOLDEN, "candidate_graph_cascade.txt")):
        if not line.strip() or line[0] == "#":
            continue
        key, *rest = line.split()
        if key == "edge":
            u, u2, entry = int(rest[0]), int(rest[1]), rest[2]
            v, lst = entry.split(":")
            d["edge"].append((u, u2, int(v), [int(x) for x in lst.split(",") if x]))
        elif key in ("round1", "final"):
            d[key] = [sorted(int(x) for x in s.split(",")) for s in rest]
        else:
            d[key] = [int(x) for x in rest]
    return d


def test_hand_worked_cascade():
    d = _golden()
    n = d["n"][0]
    e = np.array(d["edges"], dtype=np.int32).reshape(-1, 2)
    rowptr, col = gg.csr_from_edges(n, e)
    k = d["qk"][0]
    qe = np.array(d["qedges"], dtype=np.int32).reshape(-1, 2)
    c0 = CG.label_sets(np.array(d["labels"]), k, d["qlabels"], n)
    r1, rounds1 = CG.refine(rowptr, col, k, qe, c0, max_rounds=1)
    assert rounds1 == 1
    assert [sorted(np.flatnonzero(r1[u]).tolist()) for u in range(k)] == d["round1"]
    fin, rounds = CG.refine(rowptr, col, k, qe, c0)
    assert [sorted(np.flatnonzero(fin[u]).tolist()) for u in range(k)] == d["final"]
    assert rounds == d["rounds"][0]
    ce = CG.candidate_edges(rowptr, col, k, qe, fin)
    assert len(ce) == 2 * len(qe)
    for u, u2, v, lst in d["edge"]:
        vs, ptr, adj = ce[(u, u2)]
        i = int(np.flatnonzero(vs == v)[0])
        assert adj[ptr[i]:ptr[i + 1]].tolist() == lst


def _random_case(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 11))
    L = int(rng.integers(1, 4))
    g = gg.er_graph(n, float(rng.uniform(0.25, 0.6)), 100 + seed, num_labels=L)
    k = int(rng.integers(2, 6))
    edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
    rng.shuffle(pairs)
    edges |= set(pairs[:int(rng.integers(0, 3))])
    qe = np.array(sorted(edges), dtype=np.int32)
    ql = rng.integers(0, L, size=k).astype(np.int32) if L > 1 else None
    labels = g.labels if L > 1 else None
    return g, labels, L, k, qe, ql


@pytest.mark.parametrize("seed", range(40))
def test_every_embedding_lies_in_the_candidate_graph(seed):
    g, labels, L, k, qe, ql = _random_case(seed)
    n = g.n
    c0 = CG.bits_to_sets(O.filter_bits(g.rowptr, g.col, labels, L, k, qe, ql), n)
    fin, _ = CG.refine(g.rowptr, g.col, k, qe, c0)
    ce = CG.candidate_edges(g.rowptr, g.col, k, qe, fin)
    emb = O.brute(g.rowptr, g.col, labels, k, qe, ql)["rows"]
    for M in emb:
        for u in range(k):
            assert fin[u, M[u]]
        for (u, u2), (vs, ptr, adj) in ce.items():
            i = int(np.searchsorted(vs, M[u]))
            assert vs[i] == M[u] and M[u2] in adj[ptr[i]:ptr[i + 1]]
    # the search restricted to the refined sets finds the same embeddings
    full = O.match(g.rowptr, g.col, labels, k, qe, ql)
    restricted = O.match(g.rowptr, g.col, labels, k, qe, ql, cand_bits=CG.sets_to_bits(fin))
    assert (restricted["count"], restricted["hash"]) == (full["count"], full["hash"]) == \
        (len(emb), sum(O.embedding_hash(M) for M in emb) % (1 << 64))


@pytest.mark.parametrize("seed", range(40))
def test_fixed_point_has_support_and_is_order_independent(seed):
    g, labels, L, k, qe, ql = _random_case(seed)
    n = g.n
    c0 = CG.label_sets(labels, k, ql, n)
    fin, _ = CG.refine(g.rowptr, g.col, k, qe, c0)
    nb = [set() for _ in range(k)]
    for a, b in qe:
        nb[a].add(int(b))
        nb[b].add(int(a))
    adj = [set(g.neighbors(v).tolist()) for v in range(n)]
    # support condition at the fixed point, and nothing outside C_0
    for u in range(k):
        for v in range(n):
            if fin[u, v]:
                assert c0[u, v]
                assert all(any(fin[u2, x] for x in adj[v]) for u2 in nb[u])
    # in-place updates, vertices visited in descending order, until stable
    cur = c0.copy()
    changed = True
    while changed:
        changed = False
        for u in reversed(range(k)):
            for v in reversed(range(n)):
                if cur[u, v] and not all(any(cur[u2, x] for x in adj[v]) for u2 in nb[u]):
                    cur[u, v] = False
                    changed = True
    assert np.array_equal(cur, fin)


def _tree_query(rng, k, L):
    qe = np.array([(int(rng.integers(0, v)), v) for v in range(1, k)], dtype=np.int32).reshape(-1, 2)
    return qe, rng.integers(0, L, size=k).astype(np.int32)


@pytest.mark.parametrize("seed", range(30))
def test_tree_queries_refine_to_homomorphism_images(seed):
    """Arc consistency decides tree-shaped constraint problems: with
    label-only starting sets, v survives for u exactly when some
    label-preserving homomorphism (edges to edges, not necessarily
    injective) maps u to v."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 8))
    L = int(rng.integers(1, 3))
    g = gg.er_graph(n, float(rng.uniform(0.2, 0.5)), 300 + seed, num_labels=L)
    k = int(rng.integers(2, 5))
    qe, ql = _tree_query(rng, k, L)
    labels = g.labels if L > 1 else np.zeros(n, dtype=np.int32)
    adj = [set(g.neighbors(v).tolist()) for v in range(n)]
    images = np.zeros((k, n), dtype=bool)
    for h in itertools.product(range(n), repeat=k):
        if all(labels[h[u]] == ql[u] for u in range(k)) and all(h[b] in adj[h[a]] for a, b in qe):
            for u in range(k):
                images[u, h[u]] = True
    fin, _ = CG.refine(g.rowptr, g.col, k, qe, CG.label_sets(labels, k, ql, n))
    assert np.array_equal(fin, images)


def test_bitmap_round_trip_and_ragged_tail():
    rng = np.random.default_rng(3)
    for n in (1, 31, 32, 33, 70):
        s = rng.random((3, n)) < 0.4
        b = CG.sets_to_bits(s)
        assert b.shape == (3, (n + 31) // 32)
        assert np.array_equal(CG.bits_to_sets(b, n), s)


def test_empty_candidates_and_single_vertex_query():
    g = gg.er_graph(8, 0.5, 1)
    k, qe = 2, np.array([[0, 1]], dtype=np.int32)
    c0 = np.zeros((k, g.n), dtype=bool)
    c0[0, :] = True  # no candidates for u1: everything goes in one round
    fin, rounds = CG.refine(g.rowptr, g.col, k, qe, c0)
    assert not fin.any() and rounds == 1
    one, r1 = CG.refine(g.rowptr, g.col, 1, np.zeros((0, 2), np.int32), np.ones((1, g.n), bool))
    assert one.all() and r1 == 0 and CG.candidate_edges(g.rowptr, g.col, 1, np.zeros((0, 2)), one) == {}
