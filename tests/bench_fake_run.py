"""Runs bench.py's main() on the CPU with stand-ins for the CUDA calls and
for the engine, so that the JSON line each workload prints can be checked
without a GPU (test harness only: tests/test_bench_contract.py runs it in a
subprocess). The stand-in engine returns fixed, plausible statistics; the
numbers mean nothing, the keys and their types do.

usage: python tests/bench_fake_run.py <bench.py arguments>
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


_empty, _tensor = torch.empty, torch.tensor
torch.cuda.set_device = lambda *a, **k: None
torch.cuda.synchronize = lambda *a, **k: None
torch.cuda.current_stream = lambda *a, **k: None
torch.cuda.Event = _Event
torch.empty = lambda *a, device=None, **k: _empty(*a, **k)
torch.tensor = lambda *a, device=None, **k: _tensor(*a, **k)
torch.Tensor.pin_memory = lambda self, *a, **k: self

import graphgen as gg  # noqa: E402
import paper_2604_10601_gb300 as pkg  # noqa: E402
from paper_2604_10601_gb300 import sgm  # noqa: E402

_STATS = [f for f, _ in sgm.sgm_stats._fields_]


def _stats(**kw):
    st = {k: 0 for k in _STATS}
    st.update(ms_filter=0.1, ms_init=0.2, ms_search=1.5, grid_blocks=608, launches=7, list_elems=1000,
              cand_checked=1000, search_probes=50, bitmap_probes=70, task_groups=30, pool_size=100, init_depth=2,
              idle_lanes=64, scatter_rounds=40, alg_bytes=9000)
    st.update(kw)
    return st


class _Graph:
    def __init__(self, n):
        self.info = {"n": n}

    def free(self):
        pass


class _Query:
    def __init__(self, k):
        self.k, self.phi = k, list(range(k))

    def set_order(self, phi):
        self.phi = [int(x) for x in phi]

    def order_greedy(self, graph, root=None):
        self.phi = list(range(self.k)) if not root else [root] + [u for u in range(self.k) if u != root]

    def order(self):
        return np.asarray(self.phi, np.int32)

    def features(self, graph, phi=None, anchor=-1):
        return np.full((self.k, sgm.SGM_FEATURES), 0.5, np.float32)

    def order_learned(self, graph, model, beam=8, root=-1, anchor=-1):
        return dict(pred_learned=1.0, pred_greedy=2.0, used_learned=True)

    def free(self):
        pass


class _Model:
    def train(self, X, t, steps, lr):
        return np.linspace(1.0, 0.1, steps).astype(np.float32)

    def forward(self, X):
        return np.zeros(len(X), np.float32)


class _Batch:
    def __init__(self, qs):
        self.qs = qs

    def run(self, check=True):
        return dict(counts=np.array([q.k for q in self.qs], np.uint64), status=0, ms=1.0, stats=_stats(),
                    statuses=np.zeros(len(self.qs), np.int32), work=np.full(len(self.qs), 100, np.uint64))

    def free(self):
        pass


class _Engine:
    def __init__(self, device=0, stream=None):
        pass

    def load_graph(self, rowptr, col, labels=None, num_labels=1, validate=True, borrow=False):
        assert len(rowptr) >= 1 and col is not None
        return _Graph(len(rowptr) - 1)

    def query(self, k, edges, labels=None):
        return _Query(k)

    def opts(self, **kw):
        return sgm.Engine.opts(None, **kw)

    def count(self, graph, Q, want_hash=False, root_range=None, **kw):
        o = self.opts(**kw)
        lc = np.zeros(32, np.uint64)
        lc[:Q.k] = 3
        lo, hi = root_range if root_range is not None else (0, graph.info["n"])
        return {"count": (hi - lo) * Q.k, "hash": 0 if want_hash else None, "level_counts": lc,
                "stats": _stats(pool_size=min(o.tau, 5000), steals=7 if o.split_min else 0)}

    def model(self, in_dim, hidden, params):
        return _Model()

    def candidate_graph(self, graph, Q, use_filter=True, refine_rounds=0):
        eng = self

        class _CG:
            def count(self, want_hash=False, root_range=None, **kw):
                return eng.count(graph, Q, want_hash=want_hash, root_range=root_range, **kw)

            def free(self):
                pass
        return _CG()

    def batch(self, graph, queries, want_hash=False, root_ranges=None, **kw):
        self.opts(**kw)
        return _Batch(queries)


class _Clock:
    def __init__(self, index):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def summary(self):
        return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


pkg.Engine = _Engine
import bench  # noqa: E402

bench.ClockSampler = _Clock
_labelled = bench._labelled_rmat
bench._labelled_rmat = lambda scale, labels, seed: _labelled(10, labels, seed)
bench._workload_graph = lambda: gg.rmat_graph(10, 4, 0.57, 0.19, 0.19, seed=1)
bench._cfg4_graph = lambda: _labelled(10, 32, 1)
bench.CFG4_NQ = 16
if __name__ == "__main__":  # spawned worker processes import this module too
    sys.argv = ["bench.py"] + sys.argv[1:]
    bench.main()
