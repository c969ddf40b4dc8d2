"""bench.py's JSON line for every workload, produced on the CPU with
stand-ins for CUDA and the engine (tests/bench_fake_run.py): one line,
valid JSON, with the keys and types the benchmark contract asks for."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bench_fake_run.py"), *args],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def _common(d):
    for key in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "clocks"]:
        assert key in d, key
    assert d["data"] == "synthetic" and isinstance(d["config"], dict) and "workload" in d["config"]
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}


def test_default_line():
    d = _run("--steps", "2", "--warmup", "3", "--no-cpu-baseline")
    _common(d)
    assert d["metric"] == "matches/s" and d["unit"] == "matches/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["workload"] == "rmat22_ef16_zipf32_walk1024_anchored" and d["scaling"] == "weak"
    for roof in (d["roofline"], d["roofline_extension"], d["roofline_filter"]):
        assert set(roof) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
        assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
        assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-12
    assert d["roofline"] is not None and d["roofline"]["kernel"].startswith("extend_kernel")
    assert set(d["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert isinstance(d["gpu_launches"], int) and d["gpu_launches"] > 0
    assert d["counts_identical"] and d["speedup_vs_plain"] > 0 and d["query_set_ms"] == d["ms_per_step"]
    assert d["config"]["queries"] == 16 and d["learned_orders_used"] == 16
    f = d["full_set"]
    assert f["queries"] == 16 and f["unsolved_batched"] == 0 and f["solved_by_both"] == 16
    assert d["cost_model"]["rows"] > 0 and d["intersected_elements_per_s"] > 0
    assert "cpu_baseline" not in d


def test_default_line_cpu_baseline_and_reference_arm():
    d = _run("--steps", "1", "--warmup", "3", "--cpu-seconds", "1")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == "matches/s" and cb["value"] > 0
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-seconds", "1")
    assert r["impl"] == "reference" and r["metric"] == d["metric"] and r["unit"] == d["unit"]
    assert r["config"]["workload"] == d["config"]["workload"] and r["value"] > 0
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["cpu_baseline"]["cores"] >= 1


def test_pattern_line():
    d = _run("--workload", "patterns", "--steps", "2", "--warmup", "3", "--no-cpu-baseline")
    _common(d)
    assert d["metric"] == "matches/s" and d["unit"] == "matches/s" and d["higher_is_better"] is True
    assert set(d["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert abs(d["roofline"]["frac"] - d["roofline"]["achieved"] / d["roofline"]["peak"]) < 1e-12
    assert d["roofline"]["probe_sector_achieved"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["intersected_elements_per_s"] > 0
    assert abs(d["idle_rate"] - 64 / (32 * 40)) < 1e-12


@pytest.mark.parametrize("workload", ["learned", "tau"])
def test_secondary_workloads(workload):
    d = _run("--workload", workload, "--nq", "8", "--train-queries", "4", "--steps", "2", "--warmup", "3")
    _common(d)
    assert d["metric"] == "query-set time" and d["unit"] == "ms" and d["higher_is_better"] is False
    if workload == "learned":
        assert d["counts_identical"] and d["learned_orders_used"] == 8 and d["train_rows"] > 0
    else:
        assert len(d["sweep"]) == 6 and all("ms" in row for row in d["sweep"])
        assert d["value"] == d["sweep"][2]["ms"]


def test_ablation_line():
    d = _run("--workload", "ablation", "--steps", "1", "--warmup", "1", "--cap", "5")
    _common(d)
    assert d["metric"] == "query-set time" and d["higher_is_better"] is False
    assert list(d["ablation"]) == ["Naive", "Unroll-4", "Unroll-8", "Fine(naive)", "Fine(batch)"]
    fb = d["ablation"]["Fine(batch)"]
    assert d["value"] == sum(fb["patterns_ms"].values()) and fb["large_solved"] == 16
    assert d["ablation"]["Naive"]["large_speedup_vs_naive_geomean"] == 1.0


def test_cgraph_line():
    d = _run("--workload", "cgraph", "--warmup", "1", "--cap", "5")
    _common(d)
    assert d["metric"] == "query-set time" and d["counts_identical"]
    assert len(d["queries"]) == 16 and d["solved"] == {"bitmaps": 16, "cgraph": 16}
    assert abs(d["value"] - d["both_solved_ms"]["cgraph"]) < 1e-9


def test_per_query_jsonl_log(tmp_path):
    path = str(tmp_path / "runs.jsonl")
    _run("--workload", "patterns", "--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--log-jsonl", path)
    from paper_2604_10601_gb300 import runlog
    recs = runlog.read(path)
    assert [r["query"] for r in recs] == ["K4", "K5", "house5d", "house6d", "C4", "P5"]
    for r in recs:
        assert r["count"] >= 0 and r["root_range"][0] < r["root_range"][1] and r["world"] == 1
        assert r["intersected_elements"] == 1000 and r["alg_bytes"] == 9000
        assert r["probe_sector_bytes"] == 4 * 1000 + 32 * 120 + 12 * 30
        assert abs(r["idle_rate"] - 64 / (32 * 40)) < 1e-12 and len(r["level_counts"]) >= 1


def test_runlog_bytes_match_the_bench_roofline_formula():
    import bench
    from paper_2604_10601_gb300 import runlog
    st = dict(list_elems=7, search_probes=3, bitmap_probes=5, task_groups=11, alg_bytes=123)
    assert runlog.alg_bytes(st) == bench._alg_bytes(st) == 123
    assert runlog.probe_sector_bytes(st) == bench._probe_sector_bytes(st) == 4 * 7 + 32 * 8 + 12 * 11


def test_filter_byte_model_counts_the_scanned_bucket_prefixes():
    """The batched filter's byte model, against a vertex-by-vertex count of
    what the label-bucket filter reads: per query and label of its vertices,
    every vertex of that label whose degree class min(d, 8) reaches the
    smallest query degree of the label, 8 B plus one byte per distinct label
    needed by that label's query vertices; plus the bitmaps."""
    import numpy as np
    import bench
    import graphgen as gg
    g = gg.er_graph(300, 0.02, 4, num_labels=3)
    deg = np.diff(g.rowptr)
    qs = [gg.Query(4, [[0, 1], [1, 2], [2, 0], [2, 3]], [0, 1, 0, 2]),
          gg.Query(3, [[0, 1], [1, 2]], [1, 1, 1]),
          gg.Query(2, [[0, 1]], [2, 0])]
    words = (g.n + 31) // 32
    want = 0.0
    for q in qs:
        dq = np.zeros(q.k, dtype=int)
        for a, b in q.edges:
            dq[a] += 1
            dq[b] += 1
        for lab in set(int(x) for x in q.labels):
            us = [u for u in range(q.k) if q.labels[u] == lab]
            need = {int(q.labels[w]) for u in us for a, b in q.edges for w in ((b,) if a == u else (a,) if b == u else ())}
            c = min(min(dq[u] for u in us), 8)
            scanned = sum(1 for v in range(g.n) if g.labels[v] == lab and min(deg[v], 8) >= c)
            want += scanned * (8 + len(need))
        want += 4 * q.k * words
    assert bench._filter_bytes(qs, g, 3) == want
