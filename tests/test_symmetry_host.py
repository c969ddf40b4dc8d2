"""Symmetry breaking, host side (no GPU): the automorphism groups and the
stabiliser-chain constraints the engine builds, checked through the C ABI
against brute force with the CPU oracle. For every order and mode, the
embeddings that satisfy the constraints (rank = (degree, id) of the data
vertex) must number |all| / |H|, and expanding them over H must give every
embedding exactly once."""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from paper_2604_10601_gb300 import sgm

NAMES = ["K3", "K4", "C4", "C5", "P3", "P4", "S3", "house5d", "house6d", "tailed_triangle"]


def _q(name):
    return gg.pattern(name)


def _connected_orders(k, edges, limit, rng):
    adj = [set() for _ in range(k)]
    for a, b in np.asarray(edges).reshape(-1, 2):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    out = []
    for p in itertools.permutations(range(k)):
        if all(adj[p[i]] & set(p[:i]) for i in range(1, k)):
            out.append(list(p))
    if len(out) > limit:
        out = [out[i] for i in rng.choice(len(out), size=limit, replace=False)]
    return out


@pytest.mark.parametrize("name", NAMES)
def test_automorphisms_are_the_embeddings_of_q_in_itself(name):
    q = _q(name)
    rp, col = gg.csr_from_edges(q.k, q.edges)
    ref = O.match(rp, col, q.labels, q.k, q.edges, q.labels, want_rows=True)
    aut = sgm.sgm_query_automorphisms(q.k, q.edges, q.labels)
    assert len(aut) == ref["count"]
    assert np.array_equal(aut[0], np.arange(q.k))  # identity first
    # embeddings of Q in itself listed by query vertex: row[u] = sigma(u)
    assert sorted(map(tuple, aut.tolist())) == sorted(map(tuple, ref["rows"].tolist()))


def _rank(g):
    deg = g.degrees()
    order = np.lexsort((np.arange(g.n), deg))  # by degree, then id
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    return rank


@pytest.mark.parametrize("seed", range(6))
def test_constraints_pick_one_embedding_per_orbit(seed):
    rng = np.random.default_rng(300 + seed)
    nl = 1 if seed < 3 else 2
    g = gg.er_graph(int(rng.integers(14, 30)), 0.35, 40 + seed, num_labels=nl)
    rank = _rank(g)
    for name in NAMES:
        q = _q(name)
        labels = q.labels if (q.labels is None or nl > 2) else None
        if nl > 1 and labels is None:
            labels = rng.integers(0, nl, size=q.k).astype(np.int32)
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, labels, want_rows=True, cap=1 << 20)
        rows = ref["rows"]
        allset = set(map(tuple, rows.tolist()))
        for phi in _connected_orders(q.k, q.edges, 4, rng):
            for count_mode in (False, True):
                plan = sgm.sgm_query_symmetry_plan(q.k, q.edges, labels, phi, count_mode)
                gt, H = plan["sb_gt"], plan["group"]
                assert len(H) == plan["group_n"] >= 1
                keep = np.ones(len(rows), dtype=bool)
                for lvl in range(q.k):
                    for i in range(lvl):
                        if (int(gt[lvl]) >> i) & 1:
                            keep &= rank[rows[:, phi[lvl]]] > rank[rows[:, phi[i]]]
                kept = rows[keep]
                assert len(kept) * len(H) == len(rows), (name, phi, count_mode)
                expanded = {tuple(int(M[s[u]]) for u in range(q.k)) for M in kept for s in H}
                assert expanded == allset, (name, phi, count_mode)
                if plan["arith"]:
                    assert count_mode and gt[q.k - 1] == 0


def test_upper_list_levels_are_constrained_backward_neighbours():
    q = _q("K4")
    phi = [0, 1, 2, 3]
    plan = sgm.sgm_query_symmetry_plan(q.k, q.edges, None, phi, False)
    # K4: a full chain M[phi0] < M[phi1] < M[phi2] < M[phi3], every earlier
    # vertex a backward neighbour, so every constraint may use N+
    assert [int(x) for x in plan["sb_gt"]] == [0, 0b1, 0b11, 0b111]
    assert np.array_equal(plan["up"], plan["sb_gt"])
    assert plan["group_n"] == 24
    # a star in count mode: the arithmetic last level keeps H = Stab(last leaf)
    s = _q("S3")
    p = sgm.sgm_query_symmetry_plan(s.k, s.edges, None, [0, 1, 2, 3], True)
    assert p["arith"] and p["group_n"] == 2 and p["sb_gt"][3] == 0
    p = sgm.sgm_query_symmetry_plan(s.k, s.edges, None, [0, 1, 2, 3], False)
    assert not p["arith"] and p["group_n"] == 6


def test_host_query_errors():
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_query_symmetry_plan(3, [[0, 1], [1, 2]], None, [0, 2, 1])
    assert ei.value.status == sgm.SGM_E_ORDER_NOT_CONNECTED
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_query_automorphisms(2, [[0, 0]])
    assert ei.value.status == sgm.SGM_E_QUERY_INVALID
