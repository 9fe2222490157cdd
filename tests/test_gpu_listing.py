"""Clique listing (rows of vertex IDs) through the C ABI: every row is a
clique, rows are distinct as vertex sets, each row follows the DAG's
orientation order, and their number equals the oracle's count -- so the rows
are exactly the k-cliques."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu


def list_rows(g, k):
    import torch

    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        n = pgm.pgm_list_kcliques(h, k)  # size query
        buf = torch.full((max(n, 1), k), -1, dtype=torch.int32, device="cuda")
        got = pgm.pgm_list_kcliques(h, k, buf.data_ptr(), n)
        assert got == n
        return buf[:n].cpu().numpy()
    finally:
        pgm.pgm_graph_destroy(h)


def check_rows(g, k, rows):
    rp, col = np.asarray(g.rowptr), np.asarray(g.col)
    deg = np.diff(rp)
    adj = {(int(u), int(v)) for u in range(g.n) for v in col[rp[u]:rp[u + 1]]}
    seen = set()
    for r in rows:
        r = [int(x) for x in r]
        assert len(set(r)) == k
        for i in range(k):
            for j in range(i + 1, k):
                assert (r[i], r[j]) in adj
        # orientation order: (degree, id) increases along the row
        keys = [(int(deg[v]), v) for v in r]
        assert keys == sorted(keys)
        seen.add(tuple(sorted(r)))
    assert len(seen) == len(rows)


GRAPHS = [gg.complete(9), gg.barabasi_albert(600, 6, seed=31), gg.rmat(1 << 10, 8000, seed=32),
          gg.erdos_renyi(200, 0.2, seed=33), gg.complete_multipartite((4, 5, 6, 7)), gg.star(30), gg.empty(4)]


@pytest.mark.parametrize("g", GRAPHS, ids=[g.name for g in GRAPHS])
def test_list_kcliques(g):
    for k in range(1, 7):
        rows = list_rows(g, k)
        assert len(rows) == oracle.clique_count(g, k, "degree"), k
        check_rows(g, k, rows)


def test_list_chunked_and_overflow():
    import torch

    g = gg.barabasi_albert(1500, 9, seed=34)
    defaults = pgm.pgm_get_options()
    pgm.pgm_set_options(level_budget=1024)  # many edge-blocking chunks
    try:
        for k in (3, 4, 5):
            rows = list_rows(g, k)
            assert len(rows) == oracle.clique_count(g, k, "degree")
            check_rows(g, k, rows)
    finally:
        pgm.pgm_set_options(**defaults)
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        n = pgm.pgm_list_kcliques(h, 4)
        buf = torch.zeros((n - 1, 4), dtype=torch.int32, device="cuda")
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_list_kcliques(h, 4, buf.data_ptr(), n - 1)
        assert e.value.status == pgm.PGM_EOVERFLOW
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_list_kcliques(h, 11)
        assert e.value.status == pgm.PGM_EUNSUPPORTED
    finally:
        pgm.pgm_graph_destroy(h)
