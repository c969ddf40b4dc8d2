"""The multi-rank path on CPU: two gloo ranks split the root candidates by
vertex-id range, each counts its own shard, and the all-reduced sums equal
the whole count and hash. Shard results come from the CPU oracle, so this
covers the host-side sharding logic without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, names, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import graphgen as gg
    import oracle as O
    from paper_2604_10601_gb300.shard import root_range
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.rmat_graph(10, 4, seed=3)
    lo, hi = root_range(g.n, world, rank)
    res = []
    for name in names:
        q = gg.pattern(name)
        own = O.match(np.zeros(2, np.int64), np.zeros(0, np.int32), None, q.k, q.edges)["order"]
        r = O.match(g.rowptr, g.col, None, q.k, q.edges, root=(int(own[0]), lo, hi))
        # counts and hashes as int64 words: the hash sum wraps mod 2^64 like uint64
        t = torch.tensor([r["count"], np.int64(np.uint64(r["hash"]).view(np.int64))], dtype=torch.int64)
        dist.all_reduce(t)
        res.append((int(t[0]), int(t[1]) & ((1 << 64) - 1)))
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        out.put(res)


def test_root_range_partition():
    from paper_2604_10601_gb300.shard import root_range, combine
    for n in [0, 1, 7, 1000, 1 << 20]:
        for world in [1, 2, 3, 8]:
            rs = [root_range(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    with pytest.raises(ValueError):
        root_range(10, 2, 2)
    assert combine([(1, (1 << 64) - 1), (2, 3)]) == (3, 2)


def test_two_gloo_ranks_sum_to_the_whole():
    import graphgen as gg
    import oracle as O
    names = ["K3", "C4", "P4", "house5d"]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, names, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = out.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.rmat_graph(10, 4, seed=3)
    for name, (c, h) in zip(names, res):
        q = gg.pattern(name)
        full = O.match(g.rowptr, g.col, None, q.k, q.edges)
        assert (c, h) == (full["count"], full["hash"]), name
