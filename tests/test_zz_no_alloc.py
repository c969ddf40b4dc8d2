"""sgm_count_noalloc, the count entry point that allocates nothing.

It is for callers that cannot allocate device memory while a query runs: a
service whose device memory belongs to another framework's caching allocator,
a server that must not stall its other streams with cudaMalloc/cudaFree, a
deployment that reserves all of its memory at start-up. Checked through the C
ABI against the CPU oracle and against sgm_count on the same inputs: two calls
in a row on the same static scratch, different queries and graphs, that the
calls after the first one leave the device's free memory and torch's
allocator untouched, and the size limit. Collected last, so a run that stops
at the first failure has run every other test."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    rp = torch.from_numpy(g.rowptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    lab = None if g.labels is None else torch.from_numpy(g.labels).cuda()
    return rp, col, lab


def _noalloc(g, dev, q, phi=None):
    import torch
    from paper_2604_10601_gb300 import sgm
    rp, col, lab = dev
    stream = torch.cuda.current_stream().cuda_stream
    return sgm.sgm_count_noalloc(0, stream, g.n, rp.data_ptr(), col.data_ptr(),
                                 None if lab is None else lab.data_ptr(),
                                 g.num_labels if lab is not None else 1, q.k, q.edges, q.labels, phi)


def test_noalloc_matches_oracle_and_sgm_count_twice_in_a_row():
    from paper_2604_10601_gb300 import Engine
    eng = Engine(0)
    g = gg.rmat_graph(10, 4, seed=11)
    dev = _dev(g)
    G = eng.load_graph(g.rowptr, g.col)
    for name in ["K3", "C4", "house5d", "P4", "K4", "S3"]:
        q = gg.pattern(name)
        want = O.match(g.rowptr, g.col, None, q.k, q.edges)["count"]
        Q = eng.query(q.k, q.edges)
        ref = eng.count(G, Q, time_cap_s=60)["count"]
        first = _noalloc(g, dev, q)
        second = _noalloc(g, dev, q)
        assert ref == want, name
        assert first == want and second == want, name
        Q.free()
    G.free()
    # a labelled graph next: the scratch keeps the previous call's contents
    g2 = gg.er_graph(1500, 0.006, 3, num_labels=3)
    dev2 = _dev(g2)
    G2 = eng.load_graph(g2.rowptr, g2.col, g2.labels, 3)
    for q in [gg.pattern("tailed_triangle"), gg.Query(3, [[0, 1], [1, 2]], [2, 0, 1]),
              gg.Query(1, np.zeros((0, 2), np.int32), [1])]:
        want = O.match(g2.rowptr, g2.col, g2.labels, q.k, q.edges, q.labels)["count"]
        Q = eng.query(q.k, q.edges, q.labels)
        ref = eng.count(G2, Q, time_cap_s=60)["count"]
        assert ref == want
        assert _noalloc(g2, dev2, q) == want
        assert _noalloc(g2, dev2, q, phi=list(range(q.k))[::-1] if q.k == 3 else None) == want
        Q.free()
    G2.free()
    eng.close()


def test_noalloc_calls_leave_device_memory_untouched():
    """After a first call has loaded the library's module on the device (the
    one call that may place the static scratch there), further calls change
    neither the device's free memory nor torch's caching allocator."""
    import torch
    g = gg.rmat_graph(10, 4, seed=12)
    dev = _dev(g)
    qs = [gg.pattern(name) for name in ("K4", "C4", "P4")]
    warm = _noalloc(g, dev, qs[0])  # start-up call: every kernel of the path runs once
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    allocated0 = torch.cuda.memory_allocated()
    got = [_noalloc(g, dev, q) for q in qs for _ in range(2)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.cuda.memory_allocated() == allocated0
    want = [O.match(g.rowptr, g.col, None, q.k, q.edges)["count"] for q in qs]
    assert warm == want[0]
    assert got == [w for w in want for _ in range(2)]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2604_10601_gb300 import sgm
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(sgm.SgmError) as ei:
        sgm.sgm_count_noalloc(0, torch.cuda.current_stream().cuda_stream, 1 << 23, rp.data_ptr(), col.data_ptr(),
                              None, 1, 3, [[0, 1], [1, 2]])
    assert ei.value.status == sgm.SGM_E_INVALID_ARG
    assert "scratch" in str(ei.value)
