"""The allocation-free triangle count (pgm_count_triangles_noalloc), for
callers that cannot call cudaMalloc: its result on a device-resident DAG the
caller built must equal the regular entry point's (pgm_count_kcliques with
k = 3), exactly, on two calls in a row (the calls share one fixed scratch
array, so the second call must not see the first one's leftovers).

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

import graphgen as gg
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu


def degree_dag(g):
    """Out-lists of the (degree, ID) orientation, ascending IDs, as int32 CSR."""
    deg = np.diff(g.rowptr)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.col.astype(np.int64)
    keep = (deg[src] < deg[dst]) | ((deg[src] == deg[dst]) & (src < dst))
    rp = np.zeros(g.n + 1, np.int64)
    np.cumsum(np.bincount(src[keep], minlength=g.n), out=rp[1:])
    return rp.astype(np.int32), dst[keep].astype(np.int32)  # CSR order keeps lists sorted


@pytest.mark.parametrize("tiles", ["default", "small"])
def test_noalloc_matches_regular_entry_point(tiles):
    import torch

    saved = pgm.pgm_get_options()
    if tiles == "small":  # hub parents go through the fixed scratch list
        pgm.pgm_set_options(warp_stage_cap=32, hub_threshold=32)
    try:
        for g in [gg.barabasi_albert(20000, 8, seed=31), gg.rmat(1 << 14, 200000, seed=32), gg.complete(40)]:
            with pgm.Graph(g) as G:
                want = G.kcliques(3)
            rp, col = degree_dag(g)
            d_rp = torch.tensor(rp, device="cuda")
            d_col = torch.tensor(col if col.size else np.zeros(1, np.int32), device="cuda")
            out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            for _ in range(2):
                out.fill_(-1)
                pgm.pgm_count_triangles_noalloc(g.n, d_rp.data_ptr(), d_col.data_ptr(), int(col.size),
                                                out.data_ptr())
                assert int(out.item()) == want, (g.name, tiles)
    finally:
        pgm.pgm_set_options(**saved)


def test_noalloc_rejects_oversize():
    import torch

    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = out.data_ptr()  # never read: the size check comes before any device work
    with pytest.raises(pgm.PgmError) as e:
        pgm.pgm_count_triangles_noalloc(10, p, p, 1 << 31, p)
    assert e.value.status == pgm.PGM_EUNSUPPORTED


def test_noalloc_bound_follows_effective_hub_threshold():
    """The size limit uses the hub threshold the kernels apply, h =
    min(hub_threshold, warp_stage_cap): with warp_stage_cap = 32 and a larger
    hub_threshold, m = 33 * (2^20 - 2) + 32 arcs is the largest accepted
    size.  One arc more is rejected before any device work; a DAG of exactly
    that many arcs (bipartite, so no triangles) is counted."""
    import torch

    saved = pgm.pgm_get_options()
    pgm.pgm_set_options(warp_stage_cap=32, hub_threshold=4096)
    try:
        limit = 33 * ((1 << 20) - 2) + 32
        out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        p = out.data_ptr()
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_count_triangles_noalloc(10, p, p, limit + 1, p)
        assert e.value.status == pgm.PGM_EUNSUPPORTED
        S = 1 << 15  # sources, each pointing to a prefix of the same 1056 targets
        deg = np.full(S, limit // S, np.int64)
        deg[: limit % S] += 1
        rp = np.zeros(S + 1057, np.int64)
        rp[1 : S + 1] = np.cumsum(deg)
        rp[S + 1 :] = limit
        col = (S + np.arange(limit, dtype=np.int64) - np.repeat(rp[:S], deg)).astype(np.int32)
        d_rp = torch.tensor(rp.astype(np.int32), device="cuda")
        d_col = torch.from_numpy(col).to("cuda")
        pgm.pgm_count_triangles_noalloc(S + 1056, d_rp.data_ptr(), d_col.data_ptr(), limit, out.data_ptr())
        assert int(out.item()) == 0
    finally:
        pgm.pgm_set_options(**saved)
