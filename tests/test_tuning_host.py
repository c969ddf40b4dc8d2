"""Host logic of the autotuner, the query-set resampling rule and the cost
model's training-row logger, driven by fake engines (no GPU): which setting
wins, how settings that hit the time cap are skipped, that differing counts
raise, which queries the work-capped resampling rule keeps, and which rows
and targets the logger produces."""
import numpy as np
import pytest

from paper_2604_10601_gb300 import autotune, sgm, workload


class _FakeBatch:
    def __init__(self, eng, kw):
        self.eng, self.kw = eng, kw
        self.freed = False

    def run(self, check=True):
        return self.eng.batch_result(self.kw)

    def free(self):
        self.freed = True


class _FakeBatchEngine:
    """ms = f(setting); counts fixed unless a setting is marked as wrong."""

    def __init__(self, ms_of, counts, wrong=None, capped=None):
        self.ms_of, self.counts = ms_of, np.asarray(counts, dtype=np.uint64)
        self.wrong = wrong or (lambda kw: False)
        self.capped = capped or (lambda kw: False)
        self.batches = []

    def batch(self, graph, queries, root_ranges=None, time_cap_s=None, **kw):
        b = _FakeBatch(self, kw)
        self.batches.append(b)
        return b

    def batch_result(self, kw):
        if self.capped(kw):
            return dict(status=sgm.SGM_E_TIME_CAP, counts=self.counts, ms=0.0)
        c = self.counts + (1 if self.wrong(kw) else 0)
        return dict(status=sgm.SGM_OK, counts=c, ms=float(self.ms_of(kw)))


GRID = dict(chunk_words=[2, 4], warps_per_block=[4, 8], split_min=[0, 256], blocks_per_sm=[0])


def test_tune_batch_picks_the_fastest_setting_and_frees_every_batch():
    ms = lambda kw: 100 - kw["chunk_words"] * 10 - kw["warps_per_block"] + (50 if kw["split_min"] == 0 else 0)
    eng = _FakeBatchEngine(ms, [5, 7, 9])
    r = autotune.tune_batch(eng, None, [None] * 3, grid=GRID)
    assert r["best"] == dict(blocks_per_sm=0, chunk_words=4, split_min=256, warps_per_block=8)
    assert r["best_ms"] == 100 - 40 - 8
    assert len(r["table"]) == 8 and all(b.freed for b in eng.batches)


def test_tune_batch_skips_settings_that_hit_the_time_cap():
    eng = _FakeBatchEngine(lambda kw: 10.0 if kw["split_min"] == 0 else 20.0, [1],
                           capped=lambda kw: kw["split_min"] == 0)
    r = autotune.tune_batch(eng, None, [None], grid=GRID)
    assert r["best"]["split_min"] == 256 and r["best_ms"] == 20.0
    assert sum(row["ms"] == float("inf") for row in r["table"]) == 4


def test_tune_batch_raises_when_no_setting_finishes():
    eng = _FakeBatchEngine(lambda kw: 1.0, [1], capped=lambda kw: True)
    with pytest.raises(RuntimeError, match="time cap"):
        autotune.tune_batch(eng, None, [None], grid=GRID)


def test_tune_batch_raises_on_differing_counts():
    eng = _FakeBatchEngine(lambda kw: 1.0, [3, 4], wrong=lambda kw: kw["warps_per_block"] == 8)
    with pytest.raises(RuntimeError, match="counts differ"):
        autotune.tune_batch(eng, None, [None, None], grid=GRID)


class _FakeCountEngine:
    """count() of query i: its count, device times from the setting; raises
    SGM_E_TIME_CAP for capped settings and SGM_E_WORK_CAP past a work cap."""

    def __init__(self, counts, ms_of=None, capped=None, work=None):
        self.counts, self.ms_of = counts, ms_of or (lambda kw: 1.0)
        self.capped = capped or (lambda kw: False)
        self.work = work  # per-query sum of level counts
        self.calls = []
        self.freed = 0

    class _Q:
        def __init__(self, eng, i):
            self.eng, self.i = eng, i

        def order_greedy(self, graph, root=None):
            self.root = root

        def free(self):
            self.eng.freed += 1

    def query(self, k, edges, labels=None):
        return self._Q(self, len(self.calls))

    def count(self, graph, Q, root_range=None, time_cap_s=None, work_cap=None, **kw):
        i = Q.i if hasattr(Q, "i") else Q
        self.calls.append(dict(i=i, root_range=root_range, work_cap=work_cap, **kw))
        if self.capped(kw):
            raise sgm.SgmError(sgm.SGM_E_TIME_CAP, "count")
        if self.work is not None:
            if work_cap is not None and self.work[i] > work_cap:
                raise sgm.SgmError(sgm.SGM_E_WORK_CAP, "count")
            lc = np.zeros(32, dtype=np.uint64)
            lc[0] = self.work[i]
            return dict(count=self.counts[i], level_counts=lc)
        t = self.ms_of(kw)
        return dict(count=self.counts[i], stats=dict(ms_filter=0.0, ms_init=0.0, ms_search=t))


def test_tune_single_sums_device_time_over_the_queries():
    eng = _FakeCountEngine([10, 20], ms_of=lambda kw: kw["pool_chunk"] / 256 + kw["split_min"] / 1024)
    grid = dict(warps_per_block=[4], split_min=[64, 1024], pool_chunk=[256, 1024], blocks_per_sm=[0])
    r = autotune.tune_single(eng, None, [0, 1], grid=grid, root_ranges=[(0, 5), (5, 9)])
    assert r["best"] == dict(blocks_per_sm=0, pool_chunk=256, split_min=64, warps_per_block=4)
    assert np.isclose(r["best_ms"], 2 * (1 + 64 / 1024))
    assert {c["root_range"] for c in eng.calls} == {(0, 5), (5, 9)}


def test_tune_single_skips_capped_settings():
    eng = _FakeCountEngine([1], capped=lambda kw: kw["split_min"] == 64)
    grid = dict(warps_per_block=[4], split_min=[64, 256], pool_chunk=[512], blocks_per_sm=[0])
    r = autotune.tune_single(eng, None, [0], grid=grid)
    assert r["best"]["split_min"] == 256
    assert [row["ms"] for row in r["table"]] == [float("inf"), 1.0]


class _Q:
    def __init__(self, k):
        self.k, self.edges, self.labels = k, np.zeros((0, 2), dtype=np.int32), None


def test_select_bounded_keeps_queries_within_the_work_bound():
    keep = 1000
    work = [10, keep, keep + 1, 10 ** 9, 0]
    eng = _FakeCountEngine([1] * len(work), work=work)
    kept, rejected = workload.select_bounded(eng, None, [_Q(4)] * len(work), keep=keep)
    assert kept == [0, 1, 4] and rejected == [2, 3]
    assert eng.freed == len(work)  # every registered query is freed
    # the cap leaves room for the bound plus the reporting slack of any launch
    assert all(c["work_cap"] >= 2 * keep for c in eng.calls)


def test_select_bounded_passes_root_ranges_and_reraises_other_errors():
    eng = _FakeCountEngine([1, 1], work=[1, 1])
    workload.select_bounded(eng, None, [_Q(3), _Q(3)], root_ranges=[(7, 8), (9, 10)], keep=10)
    assert [c["root_range"] for c in eng.calls] == [(7, 8), (9, 10)]

    class _Failing(_FakeCountEngine):
        def count(self, *a, **kw):
            raise sgm.SgmError(sgm.SGM_E_INVALID_ARG, "count")

    with pytest.raises(sgm.SgmError):
        workload.select_bounded(_Failing([1], work=[1]), None, [_Q(3)], keep=10)


class _FakeLogQuery:
    """A query whose engine-side features are the order itself (padded)."""

    def __init__(self, eng, k):
        self.eng, self.k, self.phi, self.freed = eng, k, None, False

    def set_order(self, phi):
        self.phi = [int(x) for x in phi]

    def order_greedy(self, graph, root=None):
        self.phi = list(range(self.k)) if root is None else [root] + [u for u in range(self.k) if u != root]

    def order(self):
        return np.asarray(self.phi, dtype=np.int32)

    def features(self, graph, phi=None, anchor=-1):
        f = np.zeros((self.k, sgm.SGM_FEATURES), np.float32)
        f[:, 0] = phi
        f[:, 1] = anchor
        return f

    def free(self):
        self.freed = True


class _FakeLogEngine:
    """count(): level counts 10^(position) + phi[0]; orders starting at a
    capped vertex raise SGM_E_TIME_CAP."""

    def __init__(self, capped_first=()):
        self.capped_first = set(capped_first)
        self.calls, self.queries = [], []

    def query(self, k, edges, labels=None):
        q = _FakeLogQuery(self, k)
        self.queries.append(q)
        return q

    def count(self, graph, Q, time_cap_s=None, root_range=None, **kw):
        self.calls.append(dict(phi=list(Q.phi), root_range=root_range, **kw))
        if Q.phi[0] in self.capped_first:
            raise sgm.SgmError(sgm.SGM_E_TIME_CAP, "count")
        lc = np.zeros(32, np.uint64)
        lc[:Q.k] = [10 ** i + Q.phi[0] for i in range(Q.k)]
        return dict(count=int(lc[Q.k - 1]), level_counts=lc)


class _WalkQ:
    def __init__(self, k, source):
        self.k = k
        self.edges = np.array([[i, i + 1] for i in range(k - 1)], dtype=np.int32)  # a path
        self.labels = None
        self.source = np.arange(source, source + k)


def test_log_query_skips_capped_orders_and_logs_exact_prefix_counts():
    from paper_2604_10601_gb300 import costmodel
    eng = _FakeLogEngine(capped_first={2})
    Q = eng.query(3, None)
    X, t, works = costmodel.log_query(eng, None, Q, [[0, 1, 2], [2, 1, 0], [1, 0, 2]], anchor=None)
    assert X.shape == (6, sgm.SGM_FEATURES) and X.dtype == np.float32
    want = np.log10(1.0 + np.array([1 + 0, 10 + 0, 100 + 0, 1 + 1, 10 + 1, 100 + 1], dtype=np.float64))
    assert np.allclose(t, want.astype(np.float32))
    assert works == [111.0, 114.0]
    # counts are logged without symmetry breaking or the arithmetic last level
    assert all(c["sym_break"] == 0 and c["arith_last"] == 0 and c["root_range"] is None for c in eng.calls)


def test_log_query_all_capped_gives_no_rows():
    from paper_2604_10601_gb300 import costmodel
    eng = _FakeLogEngine(capped_first={0, 1, 2})
    X, t, works = costmodel.log_query(eng, None, eng.query(3, None), [[0, 1, 2], [1, 0, 2]])
    assert X.shape == (0, sgm.SGM_FEATURES) and t.shape == (0,) and works == []


def test_build_dataset_anchored_orders_start_at_the_anchor():
    from paper_2604_10601_gb300 import costmodel
    eng = _FakeLogEngine()
    qs = [_WalkQ(4, 100), _WalkQ(5, 200)]
    X, t = costmodel.build_dataset(eng, None, qs, orders_per_query=3, seed=4, anchored=True)
    assert X.shape == ((1 + 3) * (4 + 5), sgm.SGM_FEATURES) and t.shape == (X.shape[0],)
    assert all(c["phi"][0] == 0 for c in eng.calls)  # anchored: query vertex 0 is the root
    assert [c["root_range"] for c in eng.calls] == [(100, 101)] * 4 + [(200, 201)] * 4
    assert set(X[:, 1].tolist()) == {100.0, 200.0}  # the anchor reaches the features
    assert all(q.freed for q in eng.queries)


def test_build_dataset_of_no_queries_is_empty():
    from paper_2604_10601_gb300 import costmodel
    X, t = costmodel.build_dataset(_FakeLogEngine(), None, [], anchored=True)
    assert X.shape == (0, sgm.SGM_FEATURES) and t.shape == (0,)


class _FakeHubEngine:
    """Graphs whose hub count and run time follow SGM_HUB_MIN_DEG at load."""

    def __init__(self, ms_of, wrong_at=None, capped_at=None):
        self.ms_of, self.wrong_at, self.capped_at = ms_of, wrong_at, capped_at
        self.live = 0

    class _G:
        def __init__(self, eng, t):
            self.eng, self.t = eng, t
            self.info = {"hubs": max(0, 1000 // t)}
            eng.live += 1

        def free(self):
            self.eng.live -= 1

    def load_graph(self, rowptr, col, labels=None, num_labels=1):
        import os
        return self._G(self, int(os.environ["SGM_HUB_MIN_DEG"]))

    def count(self, G, Q, time_cap_s=None, root_range=None, **kw):
        if G.t == self.capped_at:
            raise sgm.SgmError(sgm.SGM_E_TIME_CAP, "count")
        c = 10 + Q + (1 if G.t == self.wrong_at else 0)
        return dict(count=c, stats=dict(ms_filter=0.0, ms_init=0.0, ms_search=self.ms_of(G.t)))


def test_hub_threshold_tuning_picks_the_fastest_and_restores_the_environment(monkeypatch):
    import os
    monkeypatch.setenv("SGM_HUB_MIN_DEG", "777")
    eng = _FakeHubEngine(lambda t: abs(t - 512) + 1.0)
    r = autotune.tune_hub_threshold(eng, None, None, None, 1, [0, 1, 2], thresholds=[32, 512, 4096])
    assert r["best"] == {"hub_min_deg": 512} and r["best_ms"] == 3 * 1.0
    assert [row["hubs"] for row in r["table"]] == [31, 1, 0]
    assert os.environ["SGM_HUB_MIN_DEG"] == "777" and eng.live == 0
    monkeypatch.delenv("SGM_HUB_MIN_DEG")
    autotune.tune_hub_threshold(eng, None, None, None, 1, [0], thresholds=[64])
    assert "SGM_HUB_MIN_DEG" not in os.environ


def test_hub_threshold_tuning_checks_counts_and_skips_capped_thresholds():
    eng = _FakeHubEngine(lambda t: 1.0, wrong_at=4096)
    with pytest.raises(RuntimeError, match="counts differ"):
        autotune.tune_hub_threshold(eng, None, None, None, 1, [0, 1], thresholds=[32, 4096])
    assert eng.live == 0
    eng = _FakeHubEngine(lambda t: 1.0 / t, capped_at=4096)
    r = autotune.tune_hub_threshold(eng, None, None, None, 1, [0], thresholds=[32, 4096])
    assert r["best"] == {"hub_min_deg": 32} and r["table"][1]["ms"] == float("inf")


def test_default_grids_name_engine_options():
    fields = {f for f, _ in sgm.sgm_opts._fields_}
    for grid in (autotune.DEFAULT_BATCH_GRID, autotune.DEFAULT_SINGLE_GRID):
        assert set(grid) <= fields
        assert all(len(v) >= 1 for v in grid.values())
    assert sgm.Engine.opts(None, **next(autotune._grid(autotune.DEFAULT_SINGLE_GRID))).tau == 10 ** 5
