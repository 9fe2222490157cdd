"""The N > 1 path of bench.py on CPU: two gloo ranks split the vertices with
bench.vertex_shares, count their share of the cliques (the CPU oracle stands
in for each rank's device), and sum the per-level counts with bench's own
exact reduction, bench.allreduce_u64; the sum must equal the
single-process count.  The range semantics match pgm_count_kcliques_range:
a clique belongs to the share holding its first vertex in (degree, ID) order.
A second case sums counts above 2^53 (where a float64 sum would round) and
near 2^64, bit-exactly."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import bench
    import graphgen as gg
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.barabasi_albert(4000, 9, seed=21)
    lo, hi = bench.vertex_shares(g, world)[rank]
    lv = oracle.clique_levels(g, 4, "degree", roots=(lo, hi))
    tot = bench.allreduce_u64(lv[2:5], dist)
    # large counts: rank r holds 2^53 + 1 + r and 2^63 - 1 - r; their sums need
    # 55 and 64 bits and are odd, so a float64 reduction would be off by one
    big = bench.allreduce_u64([(1 << 53) + 1 + rank, (1 << 63) - 1 - rank], dist)
    mx = bench.allreduce_max(float(rank) + 0.5, dist)
    if rank == 0:
        out.put((tot, big, mx, lo, hi))
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
    tot, big, mx, lo, hi = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.barabasi_albert(4000, 9, seed=21)
    lv = oracle.clique_levels(g, 4, "degree")
    assert tot == lv[2:5]
    assert big == [(1 << 54) + 3, (1 << 64) - 3]
    assert mx == 1.5
    assert lo == 0 and 0 < hi < g.n


def test_shares_partition():
    import bench
    import graphgen as gg

    g = gg.rmat(1 << 12, 30000, seed=3)
    for w in (1, 2, 3, 8):
        sh = bench.vertex_shares(g, w)
        assert sh[0][0] == 0 and sh[-1][1] == g.n
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))


def test_vertex_weights_are_bitset_row_work():
    """The weight of u is sum over its out-arcs u -> v of d+(v), plus d+(u) + 1
    (checked against a direct loop over a small graph's orientation)."""
    import bench
    import graphgen as gg

    g = gg.barabasi_albert(300, 4, seed=5)
    deg = np.diff(g.rowptr)
    out = [[v for v in g.col[g.rowptr[u]:g.rowptr[u + 1]] if (deg[u], u) < (deg[v], v)] for u in range(g.n)]
    want = [sum(len(out[v]) for v in out[u]) + len(out[u]) + 1 for u in range(g.n)]
    assert bench.vertex_weights(g).tolist() == want
