"""The candidate-set refinement rule of the CUDA path (csrc/refine.cuh),
built for the host with g++ and run in the engine's round structure
(tests/refine_host_check.cpp), against the candidate-graph oracle: the same
bitmaps after every number of rounds and the same count of rounds that
cleared a candidate. The GPU kernel applies this rule per vertex
(tests/test_gpu_support_refinement.py compares the kernel itself)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from oracle import candidate_graph as CG

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_10601_gb300", "csrc")


@pytest.fixture(scope="module")
def host_refine(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("refine") / "librefine_host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}",
                    os.path.join(ROOT, "tests", "refine_host_check.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.refine_host.restype = ctypes.c_int
    lib.refine_host.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 2 + [ctypes.c_int32, ctypes.c_void_p,
                                                                            ctypes.c_void_p, ctypes.c_int32]

    def run(g, k, qedges, bits, max_rounds):
        qadj = np.zeros(32, dtype=np.uint32)
        for a, b in np.asarray(qedges, dtype=np.int64).reshape(-1, 2):
            qadj[a] |= np.uint32(1) << np.uint32(b)
            qadj[b] |= np.uint32(1) << np.uint32(a)
        out = np.ascontiguousarray(bits, dtype=np.uint32).copy()
        rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
        col = np.ascontiguousarray(g.col, dtype=np.int32)
        r = lib.refine_host(g.n, rp.ctypes.data, col.ctypes.data, k, qadj.ctypes.data, out.ctypes.data, max_rounds)
        return out, r
    return run


def _case(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 300))
    L = int(rng.integers(1, 6))
    g = gg.er_graph(n, float(rng.uniform(0.01, 0.08)), 500 + seed, num_labels=L)
    k = int(rng.integers(2, 9))
    edges = {(int(rng.integers(0, v)), v) for v in range(1, k)}
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in edges]
    rng.shuffle(pairs)
    edges |= set(pairs[:int(rng.integers(0, 4))])
    qe = np.array(sorted(edges), dtype=np.int32)
    ql = rng.integers(0, L, size=k).astype(np.int32) if L > 1 else None
    return g, (g.labels if L > 1 else None), L, k, qe, ql


@pytest.mark.parametrize("seed", range(40))
def test_host_rule_matches_the_oracle_round_by_round(host_refine, seed):
    g, labels, L, k, qe, ql = _case(seed)
    for use_filter in (True, False):
        bits0 = O.filter_bits(g.rowptr, g.col, labels, L, k, qe, ql) if use_filter else \
            CG.sets_to_bits(CG.label_sets(labels, k, ql, g.n))
        c0 = CG.bits_to_sets(bits0, g.n)
        for max_rounds in (0, 1, 2, 3, 64):
            want, want_r = CG.refine(g.rowptr, g.col, k, qe, c0, max_rounds=max_rounds)
            got, got_r = host_refine(g, k, qe, bits0, max_rounds)
            assert got_r == want_r
            assert np.array_equal(got, CG.sets_to_bits(want))


def test_host_rule_on_the_hand_worked_cascade(host_refine):
    e = np.array([[0, 1], [1, 2], [3, 4], [4, 5]], dtype=np.int32)
    rowptr, col = gg.csr_from_edges(6, e)
    g = gg.Graph(rowptr, col, np.array([0, 1, 2, 0, 1, 1], dtype=np.int32), 3)
    qe = np.array([[0, 1], [1, 2]], dtype=np.int32)
    c0 = CG.label_sets(g.labels, 3, [0, 1, 2], 6)
    got, r = host_refine(g, 3, qe, CG.sets_to_bits(c0), 64)
    assert r == 2
    assert [np.flatnonzero(s).tolist() for s in CG.bits_to_sets(got, 6)] == [[0], [1], [2]]


def test_host_rule_with_a_32_vertex_query(host_refine):
    """Bit 31 of the query masks (a 32-vertex path over a long path graph)."""
    n = 40
    e = np.array([[i, i + 1] for i in range(n - 1)], dtype=np.int32)
    rowptr, col = gg.csr_from_edges(n, e)
    g = gg.Graph(rowptr, col)
    k = 32
    qe = np.array([[i, i + 1] for i in range(k - 1)], dtype=np.int32)
    c0 = np.ones((k, n), dtype=bool)
    c0[31, :] = False
    c0[31, 39] = True  # the path's last vertex may only be vertex 39
    want, want_r = CG.refine(rowptr, col, k, qe, c0)
    got, got_r = host_refine(g, k, qe, CG.sets_to_bits(c0), 1000)
    assert got_r == want_r > 0
    assert np.array_equal(got, CG.sets_to_bits(want))
