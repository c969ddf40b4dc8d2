"""The execution models of the ablation of Sec. 6.3 (Table 4) give the
oracle's counts: the fine-grained batched model (the default), the
fine-grained model without batching (one partial match per scatter round)
and Alg. 1's coarse-grained model with loop unrolling 1, 2, 4 and 8
(Sec. 2.3), on labelled and unlabelled graphs, over several BFS depths of
the initialisation phase (tau). Also: the per-model accounting that the
ablation reports (stack bytes grow with the unroll factor; the naive
fine-grained model fills fewer lanes than the batched one) and the
boundary's refusals (the coarse model counts only; batched runs take the
batched model only)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

MODELS = [("fine_batch", dict(exec_model=0)), ("fine_naive", dict(exec_model=1)),
          ("coarse_u1", dict(exec_model=2, unroll=1)), ("coarse_u2", dict(exec_model=2, unroll=2)),
          ("coarse_u4", dict(exec_model=2, unroll=4)), ("coarse_u8", dict(exec_model=2, unroll=8))]


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine
    return Engine(0)


def _cases():
    rmat = gg.rmat_graph(10, 4, 0.57, 0.19, 0.19, seed=3)
    lab = gg.Graph(rmat.rowptr, rmat.col, gg.labels_uniform(rmat.n, 4, 7), 4)
    er = gg.er_graph(3000, 0.004, 2, num_labels=3)
    eru = gg.er_graph(4000, 0.003, 5)
    return [("rmat10_K4", rmat, gg.pattern("K4")), ("er4000_C5", eru, gg.pattern("C5")),
            ("rmat10_house5d", rmat, gg.pattern("house5d")),
            ("rmat10L4_walk7", lab, gg.walk_query(lab, 7, False, 1, seed=5)),
            ("rmat10L4_walk6d", lab, gg.walk_query(lab, 6, True, 0, seed=9)),
            ("er3000L3_walk5d", er, gg.walk_query(er, 5, True, 0, seed=2)),
            ("er3000L3_walk7", er, gg.walk_query(er, 7, False, 1, seed=3))]


CASES = _cases()


@pytest.mark.parametrize("name,g,q", CASES, ids=[c[0] for c in CASES])
def test_every_model_gives_the_oracle_count(eng, name, g, q):
    want = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels)["count"]
    G = eng.load_graph(g.rowptr, g.col, g.labels, g.num_labels if g.labels is not None else 1)
    Q = eng.query(q.k, q.edges, q.labels)
    Q.order_greedy(G)
    for mname, kw in MODELS:
        for tau in (1, 64, 10 ** 6):
            r = eng.count(G, Q, tau=tau, time_cap_s=120, **kw)
            assert r["count"] == want, (mname, tau)
    G.free()


def test_model_accounting(eng):
    g = gg.rmat_graph(10, 4, 0.57, 0.19, 0.19, seed=3)
    G = eng.load_graph(g.rowptr, g.col)
    q = gg.pattern("C5")
    Q = eng.query(q.k, q.edges)
    Q.order_greedy(G)
    runs = {m: eng.count(G, Q, tau=64, sym_break=0, arith_last=0, time_cap_s=120, **kw) for m, kw in MODELS}
    counts = {r["count"] for r in runs.values()}
    assert len(counts) == 1 and counts.pop() > 0
    st = {m: r["stats"] for m, r in runs.items()}
    # the coarse stacks are warps x k x unroll x d_max int32; the per-warp
    # stack grows with the unroll factor
    dmax = int(np.diff(g.rowptr).max())
    for m in ("coarse_u1", "coarse_u2", "coarse_u4", "coarse_u8"):
        u = dict(MODELS)[m]["unroll"]
        warps = st[m]["grid_blocks"] * 8
        assert st[m]["stack_bytes"] == warps * q.k * u * dmax * 4, m
    # idle lanes: every model scans the same candidates here; batching fills lanes
    def idle(m):
        return st[m]["idle_lanes"] / (32.0 * st[m]["scatter_rounds"])
    assert idle("fine_batch") < idle("fine_naive")
    assert idle("coarse_u8") < idle("coarse_u1")
    G.free()


def test_boundary_refusals(eng):
    from paper_2604_10601_gb300 import sgm
    g = gg.er_graph(500, 0.02, 1)
    G = eng.load_graph(g.rowptr, g.col)
    q = gg.pattern("K3")
    Q = eng.query(q.k, q.edges)
    with pytest.raises(sgm.SgmError) as ei:
        eng.count(G, Q, want_hash=True, exec_model=2)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    for bad in (dict(exec_model=3), dict(exec_model=-1), dict(exec_model=2, unroll=9), dict(unroll=0)):
        with pytest.raises(sgm.SgmError) as ei:
            eng.count(G, Q, **bad)
        assert ei.value.status == sgm.SGM_E_INVALID_ARG, bad
    with pytest.raises(sgm.SgmError) as ei:
        eng.count_batch(G, [Q], exec_model=1)
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    G.free()


def test_two_level_stealing_gives_the_oracle_results(eng):
    """steal_mode = 1 (Sec. 4.3's two-level balancing: idle warps offered to
    the busy warps of their block first, the device-wide range queue second)
    changes only who runs which range: counts and hashes are the oracle's,
    with small split thresholds that make warps hand ranges over often."""
    stole = 0
    for name, g, q in CASES:
        ref = O.match(g.rowptr, g.col, g.labels, q.k, q.edges, q.labels)
        G = eng.load_graph(g.rowptr, g.col, g.labels, g.num_labels if g.labels is not None else 1)
        Q = eng.query(q.k, q.edges, q.labels)
        Q.order_greedy(G)
        for kw in (dict(tau=1, split_min=2), dict(tau=64, split_min=8), dict(split_min=2, sym_break=0, arith_last=0)):
            r = eng.count(G, Q, want_hash=True, steal_mode=1, time_cap_s=120, **kw)
            assert (r["count"], r["hash"]) == (ref["count"], ref["hash"]), (name, kw)
            stole += r["stats"]["steals"]
        G.free()
    assert stole > 0
