"""Fingerprints of the seeded workloads: SHA-256 of every generated array.

The generators are deterministic (one counter-based SplitMix64 stream,
portable C), so the same seed gives the same bytes on every host. The
manifest (graphgen/manifest.json) records those bytes' hashes for the
workloads the tests and the benchmark use; the CPU tests regenerate the
smaller ones and compare, so generator drift shows up as a failed pin.

Regenerate with:  python -m graphgen.manifest        (writes manifest.json)
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import er_graph, labels_zipf, pattern, rmat_graph, walk_query_set

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "manifest.json")


def _sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _graph_fp(g) -> dict:
    fp = {"n": int(g.n), "nnz": int(g.nnz), "rowptr": _sha(g.rowptr.astype(np.int64)),
          "col": _sha(g.col[:g.nnz].astype(np.int32))}
    if g.labels is not None:
        fp["labels"] = _sha(np.asarray(g.labels, dtype=np.int32))
    return fp


def _queries_fp(qs) -> str:
    h = hashlib.sha256()
    for q in qs:
        h.update(np.int32(q.k).tobytes())
        h.update(np.ascontiguousarray(q.edges, dtype=np.int32).tobytes())
        if q.labels is not None:
            h.update(np.ascontiguousarray(q.labels, dtype=np.int32).tobytes())
        if q.source is not None:
            h.update(np.ascontiguousarray(q.source, dtype=np.int64).tobytes())
    return h.hexdigest()


def _tiny():
    return er_graph(2000, 0.004, 1, num_labels=4)


def _rmat(scale, ef, seed, labels=0, zseed=None):
    g = rmat_graph(scale, ef, 0.57, 0.19, 0.19, seed=seed)
    if labels:
        g.labels = labels_zipf(g.n, labels, 1.0, zseed)
        g.num_labels = labels
    return g


# name -> (graph builder, query-set builder or None, size class)
WORKLOADS = {
    "tiny_er2000_4labels": (_tiny, lambda g: [pattern("tailed_triangle")], "small"),
    "rmat12_ef8_zipf8_seed21": (lambda: _rmat(12, 8, 21, 8, 21),
                                lambda g: walk_query_set(g, [6, 7, 8, 9, 10, 11] * 4, [True, False] * 12, seed=77),
                                "small"),
    "rmat20_ef16_unlabelled": (lambda: _rmat(20, 16, 1), None, "large"),
    "rmat22_ef16_zipf32": (lambda: _rmat(22, 16, 1, 32, 2), None, "large"),
    "rmat24_ef16_zipf16": (lambda: _rmat(24, 16, 3, 16, 4), None, "large"),
}


def fingerprint(name: str) -> dict:
    make_g, make_q, _ = WORKLOADS[name]
    g = make_g()
    fp = {"graph": _graph_fp(g)}
    if make_q is not None:
        fp["queries"] = _queries_fp(make_q(g))
    return fp


def main() -> None:
    out = {name: fingerprint(name) for name in WORKLOADS}
    with open(PATH, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(PATH)


if __name__ == "__main__":
    main()
