"""CPU oracle for exact subgraph matching (Definition 1, Sec. 2.1).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the engine. It shares no
code with the CUDA path. The arithmetic lives in oracle.c (plain C, single
thread), built here with gcc on first use; this module only marshals numpy
arrays.

Functions:
    match(...)        all embeddings by sequential backtracking (Alg. 1 DFS)
    brute(...)        all injective maps tested one by one (tiny graphs)
    filter_bits(...)  label / degree / neighbour-label-frequency candidate sets
    embedding_hash(M) the per-embedding 64-bit hash; mix64 its mixer
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, E_ARG, E_ORDER, E_BUDGET, E_OOM = 0, -1, -2, -3, -4

_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source. Portable flags only, so the
    same source gives the same results on x86-64 and aarch64 hosts."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp],
                   check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_mix64.restype = ctypes.c_uint64
            L.oracle_mix64.argtypes = [ctypes.c_uint64]
            L.oracle_embedding_hash.restype = ctypes.c_uint64
            L.oracle_embedding_hash.argtypes = [ctypes.c_int32, _vp]
            L.oracle_match.restype = ctypes.c_int32
            L.oracle_match.argtypes = [ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                       _vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _vp, _vp,
                                       ctypes.c_uint64, _vp, _vp, _vp, ctypes.c_uint64]
            L.oracle_own_order.restype = ctypes.c_int32
            L.oracle_own_order.argtypes = [ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32, _vp]
            L.oracle_brute.restype = ctypes.c_int32
            L.oracle_brute.argtypes = [ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                       _vp, ctypes.c_uint64, _vp, _vp]
            L.oracle_filter.restype = ctypes.c_int32
            L.oracle_filter.argtypes = [ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, _vp, _vp, _vp]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _arr(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


def mix64(z: int) -> int:
    return int(lib().oracle_mix64(z & 0xFFFFFFFFFFFFFFFF))


def embedding_hash(M) -> int:
    M = _arr(M, np.int32)
    return int(lib().oracle_embedding_hash(len(M), _p(M)))


def match(rowptr, col, labels, k, qedges, qlabels=None, order=None, root=None, cand_bits=None,
          want_rows=False, cap=None, level_counts=False, max_steps=0):
    """All embeddings of the query in the data graph (see oracle.c).

    root: None or (u, lo, hi) restricting M[u] to [lo, hi).
    Returns dict(count, hash, rows (sorted lexicographically, or None), level_counts, order).
    """
    rowptr = _arr(rowptr, np.int64)
    col = _arr(col, np.int32)
    labels = _arr(labels, np.int32)
    qe = _arr(np.asarray(qedges).reshape(-1), np.int32)
    ql = _arr(qlabels, np.int32)
    order_a = _arr(order, np.int32)
    n = len(rowptr) - 1
    m = len(qe) // 2
    cb = _arr(cand_bits, np.uint32)
    rows = None
    if want_rows:
        if cap is None:
            cap = 1 << 20
        rows = np.zeros((cap, k), dtype=np.int32)
    cnt = ctypes.c_uint64(0)
    h = ctypes.c_uint64(0)
    lc = np.zeros(k, dtype=np.uint64) if level_counts else None
    ru, rlo, rhi = (-1, 0, 0) if root is None else root
    st = lib().oracle_match(n, _p(rowptr), _p(col), _p(labels), k, m, _p(qe), _p(ql), _p(order_a), ru, rlo, rhi,
                            _p(cb), _p(rows), 0 if rows is None else cap, ctypes.byref(cnt), ctypes.byref(h),
                            _p(lc), max_steps)
    if st != OK:
        raise OracleError(st)
    out = dict(count=int(cnt.value), hash=int(h.value), level_counts=lc, rows=None)
    if rows is not None:
        r = rows[:min(cap, out["count"])]
        out["rows"] = r[np.lexsort(r.T[::-1])] if len(r) else r
        out["truncated"] = out["count"] > cap
    own = np.zeros(k, dtype=np.int32)
    lib().oracle_own_order(k, m, _p(qe), ru, _p(own))
    out["order"] = order_a if order_a is not None else own
    return out


def brute(rowptr, col, labels, k, qedges, qlabels=None, cap=1 << 16):
    """Every injective map tested against Definition 1 (n <= 64)."""
    rowptr = _arr(rowptr, np.int64)
    col = _arr(col, np.int32)
    labels = _arr(labels, np.int32)
    qe = _arr(np.asarray(qedges).reshape(-1), np.int32)
    ql = _arr(qlabels, np.int32)
    n = len(rowptr) - 1
    rows = np.zeros((cap, k), dtype=np.int32)
    cnt = ctypes.c_uint64(0)
    h = ctypes.c_uint64(0)
    st = lib().oracle_brute(n, _p(rowptr), _p(col), _p(labels), k, len(qe) // 2, _p(qe), _p(ql), _p(rows), cap,
                            ctypes.byref(cnt), ctypes.byref(h))
    if st != OK:
        raise OracleError(st)
    r = rows[:min(cap, cnt.value)]
    return dict(count=int(cnt.value), hash=int(h.value), rows=r)


def filter_bits(rowptr, col, labels, num_labels, k, qedges, qlabels=None):
    """k candidate bitmaps (uint32 words, ceil(n/32) per query vertex)."""
    rowptr = _arr(rowptr, np.int64)
    col = _arr(col, np.int32)
    labels = _arr(labels, np.int32)
    qe = _arr(np.asarray(qedges).reshape(-1), np.int32)
    ql = _arr(qlabels, np.int32)
    n = len(rowptr) - 1
    words = (n + 31) // 32
    out = np.zeros((k, words), dtype=np.uint32)
    st = lib().oracle_filter(n, _p(rowptr), _p(col), _p(labels), num_labels, k, len(qe) // 2, _p(qe), _p(ql),
                             _p(out))
    if st != OK:
        raise OracleError(st)
    return out
