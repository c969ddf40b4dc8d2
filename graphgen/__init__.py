"""Seeded synthetic inputs shared by the CPU oracle and the CUDA engine.

Input generation only: data graphs (Erdos-Renyi, R-MAT), vertex labels
(uniform, Zipf), named query patterns and random-walk queries. Nothing here
checks candidates or hashes embeddings. The heavy loops are in graphgen.c,
built on first use with gcc (no CUDA needed).

Workload recipes follow the paper's setup: R-MAT as in PaRMAT (Sec. 6.1,
Datasets), uniform labels (Sec. 6.1), Zipf labels P(l) ~ (l+1)^-alpha
(Appendix A), queries grown by random walks (Sec. 6.1, Query Sets).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.gg_rand64.restype = ctypes.c_uint64
            L.gg_rand64.argtypes = [ctypes.c_uint64] * 3
            L.gg_csr_from_edges.restype = ctypes.c_int64
            L.gg_csr_from_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i64p, _i32p]
            L.gg_er_edges.restype = ctypes.c_int64
            L.gg_er_edges.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, _i32p, _i32p,
                                      ctypes.c_int64]
            L.gg_rmat_edges.restype = None
            L.gg_rmat_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64, _i32p, _i32p]
            L.gg_labels_uniform.restype = None
            L.gg_labels_uniform.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, _i32p]
            L.gg_labels_zipf.restype = None
            L.gg_labels_zipf.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                         _i32p]
            L.gg_walk_query.restype = ctypes.c_int32
            L.gg_walk_query.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_uint64, _i32p, _i32p]
            L.gg_walk_query_bounded.restype = ctypes.c_int32
            L.gg_walk_query_bounded.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                                _i32p, _i32p]
            L.gg_num_threads.restype = ctypes.c_int32
            _lib = L
    return _lib


def rand64(seed: int, stream: int, i: int) -> int:
    return int(lib().gg_rand64(seed, stream, i))


# --------------------------------------------------------------------------
# data graphs
# --------------------------------------------------------------------------
class Graph:
    """Undirected labelled graph in sorted symmetric CSR form (host arrays).

    rowptr int64[n+1], col int32[nnz] (both directions of every edge, rows
    sorted ascending, no self-loops, no duplicates), labels int32[n] or None
    (unlabelled, i.e. one label), num_labels >= 1.
    """

    def __init__(self, rowptr, col, labels=None, num_labels=1, name=""):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.labels = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
        self.num_labels = int(num_labels)
        self.name = name

    @property
    def n(self) -> int:
        return len(self.rowptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.rowptr[v]:self.rowptr[v + 1]]


def csr_from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric sorted simple CSR from an (m, 2) edge array over [0, n)."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(1, 2 * len(e)), dtype=np.int32)
    nnz = lib().gg_csr_from_edges(n, len(e), src, dst, rowptr, col)
    if nnz < 0:
        raise ValueError(f"csr_from_edges failed ({nnz})")
    return rowptr, col[:nnz].copy()


def er_graph(n: int, p: float, seed: int, num_labels: int = 1, label_seed: int | None = None) -> Graph:
    """G(n, p): each unordered pair is an edge with probability p."""
    exp = p * n * (n - 1) / 2
    cap = int(exp + 10 * np.sqrt(exp + 1) + 64)
    src = np.zeros(cap, dtype=np.int32)
    dst = np.zeros(cap, dtype=np.int32)
    m = lib().gg_er_edges(n, p, seed, src, dst, cap)
    if m < 0:
        raise RuntimeError("ER edge buffer too small")
    rowptr, col = csr_from_edges(n, np.stack([src[:m], dst[:m]], axis=1))
    labels = None
    if num_labels > 1:
        labels = labels_uniform(n, num_labels, seed if label_seed is None else label_seed)
    return Graph(rowptr, col, labels, num_labels, name=f"er{n}_p{p}_s{seed}")


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 1) -> Graph:
    """R-MAT (PaRMAT-style): m = edge_factor * 2^scale sampled edges, symmetrised,
    self-loops and duplicates removed. Unlabelled; attach labels separately."""
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib().gg_rmat_edges(scale, m, a, b, c, seed, src, dst)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(2 * m, dtype=np.int32)
    nnz = lib().gg_csr_from_edges(n, m, src, dst, rowptr, col)
    del src, dst
    if nnz < 0:
        raise RuntimeError("rmat csr build failed")
    col = col[:nnz]
    return Graph(rowptr, col, None, 1, name=f"rmat{scale}_ef{edge_factor}_s{seed}")


def labels_uniform(n: int, num_labels: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    lib().gg_labels_uniform(n, num_labels, seed, out)
    return out


def labels_zipf(n: int, num_labels: int, alpha: float, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    lib().gg_labels_zipf(n, num_labels, alpha, seed, out)
    return out


# --------------------------------------------------------------------------
# queries
# --------------------------------------------------------------------------
class Query:
    """Query graph: k vertices, undirected edge list (m, 2), labels int32[k] or None."""

    def __init__(self, k, edges, labels=None, name="", source=None):
        self.k = int(k)
        self.edges = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        self.labels = None if labels is None else np.asarray(labels, dtype=np.int32)
        self.name = name
        self.source = source  # data vertices the query was grown from (one embedding), if any

    @property
    def m(self) -> int:
        return len(self.edges)

    def flat_edges(self) -> np.ndarray:
        return np.ascontiguousarray(self.edges.reshape(-1), dtype=np.int32)

    def __repr__(self):
        return f"Query({self.name}, k={self.k}, m={self.m})"


def pattern(name: str) -> Query:
    """Named unlabelled patterns: K<k>, C<k>, P<k> (path on k vertices),
    S<k> (star with k leaves), house5d, house6d, and 'tailed_triangle'."""
    if name.startswith("K") and name[1:].isdigit():
        k = int(name[1:])
        e = [(i, j) for i in range(k) for j in range(i + 1, k)]
        return Query(k, e, name=name)
    if name.startswith("C") and name[1:].isdigit():
        k = int(name[1:])
        e = [(i, (i + 1) % k) for i in range(k)]
        return Query(k, e, name=name)
    if name.startswith("P") and name[1:].isdigit():
        k = int(name[1:])
        e = [(i, i + 1) for i in range(k - 1)]
        return Query(k, e, name=name)
    if name.startswith("S") and name[1:].isdigit():
        leaves = int(name[1:])
        e = [(0, i) for i in range(1, leaves + 1)]
        return Query(leaves + 1, e, name=name)
    if name == "house5d":
        # square 0-1-2-3, roof apex 4 on edge {0,1}, diagonal 0-2: 5 vertices, 7 edges
        e = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 0), (4, 1), (0, 2)]
        return Query(5, e, name=name)
    if name == "house6d":
        # square 0-1-2-3 with diagonal 0-2, flat roof 4-5 with 4~0 and 5~1: 6 vertices, 8 edges
        e = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (4, 5), (4, 0), (5, 1)]
        return Query(6, e, name=name)
    if name == "tailed_triangle":
        # triangle u1-u2-u3 plus pendant u4 on u1 (ids 0..3), labels (0, 1, 2, 0)
        e = [(0, 1), (1, 2), (0, 2), (0, 3)]
        return Query(4, e, labels=[0, 1, 2, 0], name=name)
    raise KeyError(name)


def walk_query(g: Graph, k: int, dense: bool, n_extra: int, seed: int, name: str = "",
               max_degree: int | None = None, min_degree: int = 1) -> Query:
    """One random-walk query of k vertices grown from g (Sec. 6.1, Query Sets).

    dense: all edges of g among the walked vertices; sparse: the walk's
    discovery tree plus n_extra further induced edges. Labels are copied from
    the data vertices, so the walked vertices are an embedding of the query.
    min_degree, max_degree: the walk visits only vertices whose degree lies
    in [min_degree, max_degree] (defaults: any; the draws are then those of
    the unbounded walk).
    """
    verts = np.zeros(k, dtype=np.int32)
    edges = np.zeros(2 * k * k, dtype=np.int32)
    if max_degree is None and min_degree <= 1:
        m = lib().gg_walk_query(g.n, g.rowptr, g.col, k, 1 if dense else 0, n_extra, seed, verts, edges)
    else:
        hi = (1 << 62) if max_degree is None else int(max_degree)
        m = lib().gg_walk_query_bounded(g.n, g.rowptr, g.col, k, 1 if dense else 0, n_extra, seed, int(min_degree),
                                        hi, verts, edges)
    if m < 0:
        raise RuntimeError("random walk did not reach k vertices")
    labels = None if g.labels is None else g.labels[verts].astype(np.int32)
    return Query(k, edges[:2 * m].reshape(-1, 2), labels, name=name or f"walk{k}_{'d' if dense else 's'}_{seed}",
                 source=verts.copy())


def walk_query_set(g: Graph, sizes, dense_flags, seed: int, n_extra_choices=(1, 2),
                   min_dense_avg_degree: float = 3.0, max_attempts: int = 64,
                   max_degree: int | None = None, min_degree: int = 1) -> list[Query]:
    """A seeded list of walk queries, one per (size, dense) pair. Dense queries
    whose average degree is below min_dense_avg_degree are redrawn with the
    next seed; sparse ones take 1 or 2 extra edges by the seeded generator.
    min_degree and max_degree as in walk_query."""
    out = []
    for qi, (k, dense) in enumerate(zip(sizes, dense_flags)):
        for attempt in range(max_attempts):
            s = int(rand64(seed, 1000 + qi, attempt))
            n_extra = n_extra_choices[s % len(n_extra_choices)]
            q = walk_query(g, int(k), bool(dense), n_extra, s, name=f"q{qi}_k{k}_{'d' if dense else 's'}",
                           max_degree=max_degree, min_degree=min_degree)
            if not dense or 2.0 * q.m / q.k >= min_dense_avg_degree:
                break
        out.append(q)
    return out


# --------------------------------------------------------------------------
# seeded initial weights of the cost-model MLP
# --------------------------------------------------------------------------
def mlp_init(in_dim: int, hidden: int, seed: int) -> np.ndarray:
    """Packed float32 initial parameters [W1, b1, W2, b2, w3, b3] of a
    3-layer MLP: weights uniform in +-sqrt(6 / fan_in) (He et al., ICCV 2015,
    uniform form), biases zero. Drawn from the counter-based rand64 stream."""
    parts = []
    for stream, (fan_in, rows, cols) in enumerate(((in_dim, in_dim, hidden), (hidden, hidden, hidden),
                                                   (hidden, hidden, 1))):
        cnt = rows * cols
        u = np.array([rand64(seed, 7000 + stream, i) >> 11 for i in range(cnt)], dtype=np.float64) / float(1 << 53)
        bound = np.sqrt(6.0 / fan_in)
        parts.append(((2.0 * u - 1.0) * bound).astype(np.float32))
        parts.append(np.zeros(cols, dtype=np.float32))
    return np.concatenate(parts)
