"""Host-side helpers of the package (no GPU): random connected orders for
the cost model's training rows, anchored root ranges, the prediction-error
summary, and the shard arithmetic."""
import numpy as np

import graphgen as gg
from paper_2604_10601_gb300 import costmodel, shard, workload


def test_random_connected_orders_are_connected_permutations():
    rng = np.random.default_rng(5)
    for name in ["K4", "C5", "P5", "house6d", "S3"]:
        q = gg.pattern(name)
        adj = costmodel._adjacency(q.k, q.edges)
        for root in (None, 0, q.k - 1):
            for _ in range(20):
                phi = costmodel.random_connected_order(q.k, adj, rng, root)
                assert sorted(phi) == list(range(q.k))
                if root is not None:
                    assert phi[0] == root
                assert all(adj[phi[i]] & set(phi[:i]) for i in range(1, q.k))


def test_random_orders_cover_every_start():
    q = gg.pattern("P4")
    adj = costmodel._adjacency(q.k, q.edges)
    rng = np.random.default_rng(1)
    starts = {costmodel.random_connected_order(q.k, adj, rng)[0] for _ in range(200)}
    assert starts == set(range(q.k))


def test_anchored_ranges_are_the_walk_sources():
    g = gg.rmat_graph(10, 4, seed=3)
    qs = gg.walk_query_set(g, [4, 5, 6], [True, False, True], seed=9)
    assert workload.anchored_ranges(qs) == [(int(q.source[0]), int(q.source[0]) + 1) for q in qs]


class _FakeModel:
    def __init__(self, y):
        self.y = np.asarray(y, dtype=np.float32)

    def forward(self, X):
        return self.y


def test_prediction_error_summary():
    err = costmodel.prediction_error(_FakeModel([1.0, 2.0, 4.0]), np.zeros((3, 2)), [1.0, 1.0, 1.0])
    assert err["rows"] == 3
    assert np.isclose(err["mae"], (0 + 1 + 3) / 3)
    assert np.isclose(err["rmse"], np.sqrt((0 + 1 + 9) / 3))


def test_shard_hash_sum_wraps():
    m = (1 << 64) - 1
    assert shard.combine([(2, m), (3, m), (0, 2)]) == (5, (2 * m + 2) & m)
