"""Host logic of the autotuner and of the query-set resampling rule, driven
by fake engines (no GPU): which setting wins, how settings that hit the
time cap are skipped, that differing counts raise, and which queries the
work-capped resampling rule keeps."""
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
