"""Full-graph counts of the pattern workload tied to closed forms, in the
settings the benchmark times (symmetry breaking on over full root ranges):

* K3 on the whole R-MAT scale-20 graph = 6 x its triangles, counted by an
  independent degree-oriented CPU count (tests/closed_forms.c);
* C4 on the whole R-MAT scale-16 graph = tr(A^4) - 2 sum d^2 + 2|E|;
* K4 on R-MAT scale 16: the symmetry-broken full-range count, the count
  without symmetry breaking, and the sum over a partition of the root range
  in the sharding mode (sym_break = 2) all agree.
Each closed form is itself pinned on small graphs (test_oracle_pins.py)."""
import numpy as np
import pytest

import closed_forms as CF
import graphgen as gg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def eng():
    from paper_2604_10601_gb300 import Engine
    return Engine(0)


def test_rmat20_triangles_against_the_degree_oriented_count(eng):
    g = gg.rmat_graph(20, 16, 0.57, 0.19, 0.19, seed=1)
    want = 6 * CF.triangles(g.rowptr, g.col)
    G = eng.load_graph(g.rowptr, g.col)
    q = gg.pattern("K3")
    Q = eng.query(q.k, q.edges)
    Q.order_greedy(G)
    assert eng.count(G, Q, time_cap_s=300)["count"] == want
    assert eng.count(G, Q, sym_break=0, time_cap_s=300)["count"] == want
    G.free()


def test_rmat16_four_cycles_against_the_trace_formula(eng):
    g = gg.rmat_graph(16, 16, 0.57, 0.19, 0.19, seed=1)
    want = CF.c4_embeddings(g.rowptr, g.col)
    G = eng.load_graph(g.rowptr, g.col)
    q = gg.pattern("C4")
    Q = eng.query(q.k, q.edges)
    Q.order_greedy(G)
    for kw in [dict(), dict(sym_break=0), dict(arith_last=0)]:
        assert eng.count(G, Q, time_cap_s=300, **kw)["count"] == want, kw
    G.free()


def test_rmat16_k4_symmetry_breaking_modes_agree(eng):
    g = gg.rmat_graph(16, 16, 0.57, 0.19, 0.19, seed=1)
    G = eng.load_graph(g.rowptr, g.col)
    q = gg.pattern("K4")
    Q = eng.query(q.k, q.edges)
    Q.order_greedy(G)
    full = eng.count(G, Q, time_cap_s=300)
    assert full["stats"]["aut_size"] == 24
    plain = eng.count(G, Q, sym_break=0, time_cap_s=300)["count"]
    cuts = np.linspace(0, g.n, 5).astype(np.int64)
    shards = sum(eng.count(G, Q, root_range=(int(a), int(b)), sym_break=2, time_cap_s=300)["count"]
                 for a, b in zip(cuts[:-1], cuts[1:]))
    assert full["count"] == plain == shards
    assert full["count"] % 24 == 0 and full["count"] > 0
    G.free()
