"""Host-side prefix features of the cost model, through the C ABI (no GPU):
values checked by hand on small queries, and the error codes."""
import math

import numpy as np
import pytest

from paper_2604_10601_gb300 import sgm


def _stats(n=1024, nnz=8192, fracs=(0.5, 0.25, 0.25), moments=(3.0, 7.0, 12.0, 18.0)):
    st = sgm.sgm_graph_stats()
    st.n, st.nnz, st.num_labels = n, nnz, len(fracs)
    for i, f in enumerate(fracs):
        st.label_frac[i] = f
    for j, m in enumerate(moments):
        st.log2_deg_moment[j] = m
    for b in range(8):
        st.deg_hist[b] = (b + 1) / 36.0
    return st


def test_tailed_triangle_prefix_features_by_hand():
    st = _stats()
    # triangle 0-1-2 plus pendant 3 on 0; labels (0, 1, 2, 0); order 0, 1, 2, 3
    f = sgm.sgm_features_from_stats(st, 4, [[0, 1], [1, 2], [0, 2], [0, 3]], [0, 1, 2, 0], [0, 1, 2, 3])
    assert f.shape == (4, sgm.SGM_FEATURES)
    sel = {0: 1.0, 1: 2.0, 2: 2.0}          # -log2 of 0.5, 0.25, 0.25
    # not anchored: feature 0 is zero; anchored at a vertex of degree 7 it is log2(8) / 32
    assert np.allclose(f[:, 0], 0.0)
    fa = sgm.sgm_features_from_stats(st, 4, [[0, 1], [1, 2], [0, 2], [0, 3]], [0, 1, 2, 0], [0, 1, 2, 3], 7)
    assert np.allclose(fa[:, 0], 3.0 / 32) and np.allclose(fa[:, 1:], f[:, 1:])
    # prefix sizes, edges, cycle rank
    assert np.allclose(f[:, 1] * 32, [1, 2, 3, 4])
    assert np.allclose(f[:, 2] * 64, [0, 1, 3, 4])
    assert np.allclose(f[:, 3] * 32, [0, 0, 1, 1])
    # new vertex: query degree, backward neighbours, selectivity
    assert np.allclose(f[:, 4] * 32, [3, 2, 2, 1])
    assert np.allclose(f[:, 5] * 32, [0, 1, 2, 1])
    assert np.allclose(f[:, 6] * 16, [sel[0], sel[1], sel[2], sel[0]])
    assert np.allclose(f[:, 7] * 128, [1, 3, 5, 6])
    # prefix-degree counts (1, 2, 3, >=4) after each step
    assert np.allclose(f[3, 8:12] * 32, [1, 2, 1, 0])      # degrees 3, 2, 2, 1
    assert np.allclose(f[1, 8:12] * 32, [2, 0, 0, 0])
    # moment term: sum over prefix vertices of log2 E[d^deg_P]
    assert np.isclose(f[3, 12] * 256, 12.0 + 7.0 + 7.0 + 3.0, rtol=1e-6)
    # graph block
    assert np.isclose(f[0, 13] * 32, 10.0) and np.isclose(f[0, 14] * 32, 13.0)
    assert np.allclose(f[0, 15:19] * np.array([16, 32, 48, 64]), [3, 7, 12, 18])
    assert np.isclose(f[0, 19] * 8, 1.5)                     # entropy of (1/2, 1/4, 1/4)
    assert np.isclose(f[0, 20] * 64, 3) and np.isclose(f[0, 21], 0.5)
    assert np.isclose(f[0, 22] * 32, 4) and np.isclose(f[0, 23] * 64, 4)
    assert np.allclose(f[0, 24:32], [(b + 1) / 36.0 for b in range(8)])
    # every row carries the same graph block
    assert np.allclose(f[:, 13:], f[0, 13:])


def test_features_depend_on_the_prefix_set_and_last_vertex_only():
    st = _stats()
    e = [[0, 1], [1, 2], [2, 3], [3, 0], [0, 2]]
    a = sgm.sgm_features_from_stats(st, 4, e, None, [0, 1, 2, 3])
    b = sgm.sgm_features_from_stats(st, 4, e, None, [1, 0, 2, 3])
    # the prefixes {0,1,2} coincide, and so does the new vertex 2
    assert np.allclose(a[2], b[2]) and np.allclose(a[3], b[3])


def test_unknown_label_has_selectivity_log2_n():
    st = _stats(n=1024)
    f = sgm.sgm_features_from_stats(st, 2, [[0, 1]], [0, 7], [0, 1])
    assert math.isclose(f[1, 6] * 16, 10.0, rel_tol=1e-6)


def test_feature_errors():
    st = _stats()
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_features_from_stats(st, 3, [[0, 1], [1, 2]], None, [0, 2, 1])
    assert ei.value.status == sgm.SGM_E_ORDER_NOT_CONNECTED
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_features_from_stats(st, 3, [[0, 1], [1, 2]], None, [0, 0, 1])
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
