"""CPU oracle for the candidate graph G' (TEST INFRASTRUCTURE ONLY).

Imported by the tests only, never by the engine; it shares no code with the
CUDA path. Plain numpy, with Python loops over vertices (small graphs).

The paper's large-query workloads (Sec. 6.1, Methods Under Study; App. C,
workload patterns) search on a candidate graph G' that a
lightweight filtering phase builds from labels and query structure, as
EGSM does, instead of on G. The paper does not define G' further. This
module takes the usual reading of such a structure:

  Candidate sets. C_0(u) is the filter's candidate set of query vertex u
  (label, degree, neighbour-label frequency; any sound superset works).
  One refinement round keeps v in C(u) only if, for every query neighbour
  u' of u, v has at least one data neighbour in C(u'):

      C_{r+1}(u) = { v in C_r(u) : N(v) ∩ C_r(u') != {} for all u' in N_Q(u) }

  (every set of round r+1 is computed from the sets of round r). The rounds
  stop at the first r with C_{r+1} = C_r, the greatest family of subsets of
  the C_0(u) closed under this support condition.

  Candidate edges. For every query edge {u, u'} and each direction u -> u',
  and every v in C(u), the sorted list N(v) ∩ C(u').

Every embedding M (Definition 1) satisfies M[u] in C(u) for every u and
M[u'] in N(M[u]) ∩ C(u') for every query edge, so searching G' instead of
G finds the same embeddings.
"""
from __future__ import annotations

import numpy as np


def _query_neighbours(k, qedges):
    nb = [set() for _ in range(k)]
    for a, b in np.asarray(qedges, dtype=np.int64).reshape(-1, 2):
        nb[int(a)].add(int(b))
        nb[int(b)].add(int(a))
    return [sorted(s) for s in nb]


def bits_to_sets(bits, n):
    """uint32 bitmaps [k, ceil(n/32)] -> bool [k, n]."""
    bits = np.asarray(bits, dtype=np.uint32)
    out = np.zeros((bits.shape[0], n), dtype=bool)
    for v in range(n):
        out[:, v] = (bits[:, v >> 5] >> np.uint32(v & 31)) & np.uint32(1)
    return out


def sets_to_bits(sets):
    """bool [k, n] -> uint32 bitmaps [k, ceil(n/32)]."""
    sets = np.asarray(sets, dtype=bool)
    k, n = sets.shape
    out = np.zeros((k, (n + 31) // 32), dtype=np.uint32)
    for v in range(n):
        out[:, v >> 5] |= sets[:, v].astype(np.uint32) << np.uint32(v & 31)
    return out


def refine_round(rowptr, col, qnb, cand):
    """One round: a new bool [k, n] from `cand` (not modified)."""
    k, n = cand.shape
    nxt = cand.copy()
    for u in range(k):
        for v in np.flatnonzero(cand[u]):
            nbrs = col[rowptr[v]:rowptr[v + 1]]
            for u2 in qnb[u]:
                if not cand[u2][nbrs].any():
                    nxt[u, v] = False
                    break
    return nxt


def refine(rowptr, col, k, qedges, cand, max_rounds=None):
    """Refined candidate sets (bool [k, n]) and the number of rounds that
    removed at least one candidate."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    cur = np.asarray(cand, dtype=bool).copy()
    qnb = _query_neighbours(k, qedges)
    rounds = 0
    while max_rounds is None or rounds < max_rounds:
        nxt = refine_round(rowptr, col, qnb, cur)
        if np.array_equal(nxt, cur):
            break
        cur = nxt
        rounds += 1
    return cur, rounds


def candidate_edges(rowptr, col, k, qedges, cand):
    """{(u, u2): (vs, ptr, adj)} for every query edge in both directions:
    vs = the vertices of C(u) ascending, adj[ptr[i]:ptr[i+1]] = the sorted
    list N(vs[i]) ∩ C(u2)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    cand = np.asarray(cand, dtype=bool)
    out = {}
    for a, b in np.asarray(qedges, dtype=np.int64).reshape(-1, 2):
        for u, u2 in ((int(a), int(b)), (int(b), int(a))):
            vs = np.flatnonzero(cand[u])
            ptr = np.zeros(len(vs) + 1, dtype=np.int64)
            lists = []
            for i, v in enumerate(vs):
                nbrs = col[rowptr[v]:rowptr[v + 1]]
                keep = np.sort(nbrs[cand[u2][nbrs]])
                lists.append(keep)
                ptr[i + 1] = ptr[i] + len(keep)
            adj = np.concatenate(lists).astype(np.int32) if lists else np.zeros(0, dtype=np.int32)
            out[(u, u2)] = (vs.astype(np.int32), ptr, adj)
    return out


def label_sets(labels, k, qlabels, n):
    """C_0 by label equality alone (bool [k, n]); unlabelled: everything."""
    if labels is None or qlabels is None:
        return np.ones((k, n), dtype=bool)
    labels = np.asarray(labels)
    return np.stack([labels == int(qlabels[u]) for u in range(k)])
