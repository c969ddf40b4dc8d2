"""Training data and training loop of the learned matching order.

The engine logs, for every prefix phi[0..i] of the order it ran, the number
of partial matches over that prefix (sgm_count's level_counts, taken with
symmetry breaking and the arithmetic last level off, so each level holds the
exact number of filtered prefix embeddings). Each prefix becomes one
training row: the SGM_FEATURES prefix features (computed in libsgm) and the
target log10(1 + count). Training runs in libsgm's MLP kernels
(sgm_model_train); this module only gathers rows and passes arrays.
"""
from __future__ import annotations

import numpy as np

from . import sgm

LOG_OPTS = dict(sym_break=0, arith_last=0)


def random_connected_order(k: int, adj: list[set], rng: np.random.Generator, root=None) -> list[int]:
    """A uniformly chosen start (or `root`), then repeatedly a uniformly chosen frontier vertex."""
    order = [int(rng.integers(0, k)) if root is None else int(root)]
    seen = {order[0]}
    while len(order) < k:
        frontier = sorted({w for u in order for w in adj[u]} - seen)
        u = int(frontier[int(rng.integers(0, len(frontier)))])
        order.append(u)
        seen.add(u)
    return order


def _adjacency(k, edges):
    adj = [set() for _ in range(k)]
    for a, b in np.asarray(edges, dtype=np.int64).reshape(-1, 2):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    return adj


def log_query(engine, graph, query, orders, time_cap_s=10.0, anchor=None, work_cap=0):
    """Runs `query` once per order and returns (features, targets, works) for
    the orders that finished within the time cap (and the work cap, in
    candidate checks, when given): features (rows, F) and targets (rows,)
    over all prefixes, works = total partial matches per order. With
    `anchor` (a data vertex), M[phi[0]] is fixed to it: the orders must all
    start at the query vertex that is anchored."""
    feats, targs, works = [], [], []
    rr = None if anchor is None else (int(anchor), int(anchor) + 1)
    for phi in orders:
        query.set_order(phi)
        try:
            r = engine.count(graph, query, time_cap_s=time_cap_s, root_range=rr, work_cap=work_cap, **LOG_OPTS)
        except sgm.SgmError as e:
            if e.status in (sgm.SGM_E_TIME_CAP, sgm.SGM_E_WORK_CAP):
                continue
            raise
        lc = np.asarray(r["level_counts"][:query.k], dtype=np.float64)
        feats.append(query.features(graph, phi, -1 if anchor is None else int(anchor)))
        targs.append(np.log10(1.0 + lc))
        works.append(float(lc.sum()))
    if not feats:
        return np.zeros((0, sgm.SGM_FEATURES), np.float32), np.zeros(0, np.float32), []
    return (np.concatenate(feats).astype(np.float32), np.concatenate(targs).astype(np.float32), works)


def build_dataset(engine, graph, queries, orders_per_query=4, seed=0, time_cap_s=10.0, include_greedy=True,
                  anchored=False, work_cap=0):
    """Training rows from each query run along its greedy order and along
    `orders_per_query` random connected orders. anchored: walk queries counted
    with their query vertex 0 fixed to the walk's source vertex. Runs past
    the time or work cap give no rows."""
    rng = np.random.default_rng(seed)
    X, t = [], []
    for q in queries:
        Q = engine.query(q.k, q.edges, q.labels)
        adj = _adjacency(q.k, q.edges)
        root = 0 if anchored else None
        anchor = int(q.source[0]) if anchored else None
        orders = []
        if include_greedy:
            Q.order_greedy(graph, root=root)
            orders.append([int(x) for x in Q.order()])
        orders += [random_connected_order(q.k, adj, rng, root) for _ in range(orders_per_query)]
        f, y, _ = log_query(engine, graph, Q, orders, time_cap_s, anchor, work_cap)
        X.append(f)
        t.append(y)
        Q.free()
    if not X:  # no queries: no rows
        return np.zeros((0, sgm.SGM_FEATURES), np.float32), np.zeros(0, np.float32)
    return np.concatenate(X), np.concatenate(t)


def train(engine, X, t, steps=2000, lr=2e-3, hidden=128, init=None):
    """A new model trained by full-batch Adam on (X, t); returns (model, losses)."""
    if init is None:
        raise ValueError("initial parameters are required (e.g. from a seeded generator)")
    m = engine.model(X.shape[1], hidden, init)
    losses = m.train(X, t, steps, lr)
    return m, losses


def prediction_error(model, X, t) -> dict:
    """Mean absolute and root-mean-square error of the predicted log10 counts."""
    y = model.forward(X)
    d = y.astype(np.float64) - np.asarray(t, np.float64)
    return dict(mae=float(np.abs(d).mean()), rmse=float(np.sqrt((d * d).mean())), rows=len(d))
