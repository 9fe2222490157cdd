"""The N > 1 path of bench.py on CPU: two gloo ranks split the vertices with
bench.vertex_shares, count their share of the cliques (the CPU oracle stands
in for each rank's device), and all-reduce the counts; the sum must equal the
single-process count.  The range semantics match pgm_count_kcliques_range:
a clique belongs to the share holding its first vertex in (degree, ID) order."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch

    import bench
    import graphgen as gg
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.barabasi_albert(4000, 9, seed=21)
    lo, hi = bench.vertex_shares(g, world)[rank]
    lv = oracle.clique_levels(g, 4, "degree", roots=(lo, hi))
    t = torch.tensor([lv[3], lv[4]], dtype=torch.int64)
    dist.all_reduce(t)
    if rank == 0:
        out.put((t.tolist(), lo, hi))
    dist.destroy_process_group()


def test_two_rank_shares_sum_to_whole():
    import graphgen as gg
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, lo, hi = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.barabasi_albert(4000, 9, seed=21)
    lv = oracle.clique_levels(g, 4, "degree")
    assert got == [lv[3], lv[4]]
    assert lo == 0 and 0 < hi < g.n


def test_shares_partition():
    import bench
    import graphgen as gg

    g = gg.rmat(1 << 12, 30000, seed=3)
    for w in (1, 2, 3, 8):
        sh = bench.vertex_shares(g, w)
        assert sh[0][0] == 0 and sh[-1][1] == g.n
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
