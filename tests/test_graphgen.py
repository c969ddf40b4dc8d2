"""The seeded input generators: determinism, CSR well-formedness, and the
label distributions they are meant to draw (Sec. 6.1; Appendix A)."""
import numpy as np
import pytest

import graphgen as gg


def _check_csr(g):
    rp, col = g.rowptr, g.col
    assert rp[0] == 0 and rp[-1] == len(col)
    assert np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert np.all(col >= 0) and np.all(col < g.n)
    assert not np.any(src == col), "self-loop"
    key = src.astype(np.int64) * g.n + col
    assert np.all(np.diff(key) > 0), "rows not strictly sorted"
    rev = col.astype(np.int64) * g.n + src
    assert np.array_equal(np.sort(rev), key), "not symmetric"


def test_rmat_deterministic_and_well_formed():
    a = gg.rmat_graph(12, 16, seed=1)
    b = gg.rmat_graph(12, 16, seed=1)
    c = gg.rmat_graph(12, 16, seed=2)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    assert not np.array_equal(a.col[:1000], c.col[:1000])
    _check_csr(a)
    # skew: vertex 0 collects the a-quadrant mass, so it is the top hub
    assert np.argmax(a.degrees()) == 0


def test_er_well_formed_and_density():
    g = gg.er_graph(2000, 0.004, 1, num_labels=4)
    _check_csr(g)
    m = g.nnz // 2
    exp = 0.004 * 2000 * 1999 / 2
    assert abs(m - exp) < 5 * np.sqrt(exp)
    freq = np.bincount(g.labels, minlength=4) / g.n
    assert np.all(np.abs(freq - 0.25) < 0.04)


def test_zipf_frequencies():
    n, L = 1 << 18, 16
    lab = gg.labels_zipf(n, L, 1.0, 3)
    p = np.array([(l + 1) ** -1.0 for l in range(L)])
    p /= p.sum()
    freq = np.bincount(lab, minlength=L) / n
    assert np.all(np.abs(freq - p) < 5 * np.sqrt(p * (1 - p) / n) + 1e-4)


def test_csr_from_edges_dedupes():
    rp, col = gg.csr_from_edges(4, [(0, 1), (1, 0), (0, 1), (2, 2), (3, 2)])
    assert rp.tolist() == [0, 1, 2, 3, 4]
    assert col.tolist() == [1, 0, 3, 2]


def test_walk_query_shape():
    g = gg.rmat_graph(12, 16, seed=4)
    g.labels = gg.labels_zipf(g.n, 16, 1.0, 4)
    for dense in (True, False):
        q = gg.walk_query(g, 12, dense, 2, 77)
        assert q.k == 12 and len(set(q.source.tolist())) == 12
        # connected
        seen, frontier = {0}, [0]
        adj = {i: set() for i in range(q.k)}
        for a, b in q.edges:
            adj[a].add(b)
            adj[b].add(a)
        while frontier:
            x = frontier.pop()
            for y in adj[x] - seen:
                seen.add(y)
                frontier.append(y)
        assert len(seen) == q.k
        if not dense:
            assert q.m <= q.k - 1 + 2
        assert np.array_equal(q.labels, g.labels[q.source])


@pytest.mark.parametrize("name", ["tiny_er2000_4labels", "rmat12_ef8_zipf8_seed21", "rmat20_ef16_unlabelled"])
def test_workloads_match_the_manifest(name):
    """The seeded workloads regenerate byte for byte (graphgen/manifest.json,
    written by python -m graphgen.manifest)."""
    import json
    from graphgen import manifest
    want = json.load(open(manifest.PATH))[name]
    assert manifest.fingerprint(name) == want
