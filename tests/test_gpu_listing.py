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


def test_list_kcliques_to_host():
    """Rows streamed to host memory through the staging buffers equal the
    device listing; a small level budget forces many chunks and flushes."""
    import torch

    g = gg.barabasi_albert(1500, 9, seed=34)
    defaults = pgm.pgm_get_options()
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        for k in (1, 2, 3, 4, 5):
            dev = list_rows(g, k)
            n = pgm.pgm_list_kcliques_host(h, k)
            out = np.full((n, k), -1, np.int32)
            assert pgm.pgm_list_kcliques_host(h, k, out) == n == len(dev)
            assert sorted(map(tuple, out)) == sorted(map(tuple, dev)), k
        pgm.pgm_set_options(level_budget=1024)
        for k in (3, 4):
            n = pgm.pgm_list_kcliques_host(h, k)
            out = torch.full((n, k), -1, dtype=torch.int32).pin_memory().numpy()
            assert pgm.pgm_list_kcliques_host(h, k, out) == n == oracle.clique_count(g, k, "degree")
            check_rows(g, k, out)
        small = np.zeros((n - 1, 4), np.int32)
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_list_kcliques_host(h, 4, small)
        assert e.value.status == pgm.PGM_EOVERFLOW
    finally:
        pgm.pgm_set_options(**defaults)
        pgm.pgm_graph_destroy(h)


# ------------------------------------------------------------ motif listing
PAIRS = [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (3, 4)]


def _class_of_code():
    """Pattern index of every 10-bit code of 5 positions, from the oracle's
    canonical class codes (minimum code over the 120 relabellings)."""
    import itertools

    index = {c: i for i, c in enumerate(oracle.p5_classes())}
    table = {}
    for code in range(1024):
        best = None
        for p in itertools.permutations(range(5)):
            c = 0
            for i, (a, b) in enumerate(PAIRS):
                if code >> i & 1:
                    x, y = sorted((p[a], p[b]))
                    c |= 1 << PAIRS.index((x, y))
            best = c if best is None else min(best, c)
        table[code] = index.get(best, -1)
    return table


def list_motif_rows(g, k):
    import torch

    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        n = pgm.pgm_list_motifs(h, k)  # size query
        buf = torch.full((max(n, 1), k + 1), -7, dtype=torch.int32, device="cuda")
        assert pgm.pgm_list_motifs(h, k, buf.data_ptr(), n) == n
        return buf[:n].cpu().numpy()
    finally:
        pgm.pgm_graph_destroy(h)


def check_motif_rows(g, k, rows, cls5):
    """Every row: a connected k-set in breadth-first canonical order (minimum
    first, then the unused vertex adjacent to the prefix with the smallest
    (first-neighbour index, ID)), labelled with its pattern; sets distinct."""
    rp, col = np.asarray(g.rowptr), np.asarray(g.col)
    adj = {(int(u), int(v)) for u in range(g.n) for v in col[rp[u]:rp[u + 1]]}
    seen = set()
    hist = [0] * {3: 2, 4: 6, 5: 21}[k]
    for r in rows:
        vs, c = [int(x) for x in r[:k]], int(r[k])
        assert len(set(vs)) == k
        order, rest = [min(vs)], set(vs) - {min(vs)}
        while rest:
            keys = [(min(i for i, w in enumerate(order) if (w, u) in adj), u) for u in rest
                    if any((w, u) in adj for w in order)]
            assert keys, r  # disconnected
            u = min(keys)[1]
            order.append(u)
            rest.remove(u)
        assert vs == order, r
        code = sum(1 << i for i, (a, b) in enumerate(PAIRS) if b < k and (vs[a], vs[b]) in adj)
        if k == 5:
            want = cls5[code]
        else:
            e = bin(code).count("1")
            dmax = max(sum(1 for i, (a, b) in enumerate(PAIRS) if code >> i & 1 and x in (a, b)) for x in range(k))
            want = e - 2 if k == 3 else {3: 0 if dmax == 3 else 1, 4: 2 if dmax == 3 else 3, 5: 4, 6: 5}[e]
        assert c == want, r
        hist[c] += 1
        seen.add(frozenset(vs))
    assert len(seen) == len(rows)
    return hist


MOTIF_GRAPHS = [gg.complete(7), gg.star(6), gg.cycle(9), gg.path(10), gg.complete_multipartite((2, 3, 3)),
                gg.from_edges(9, [(0, 1), (1, 2), (2, 0), (3, 4), (5, 6), (6, 7), (7, 8), (8, 5), (5, 7)]),
                gg.erdos_renyi(45, 0.12, seed=35), gg.barabasi_albert(60, 2, seed=36), gg.empty(3)]


@pytest.mark.parametrize("k", [3, 4, 5])
def test_list_motifs(k):
    cls5 = _class_of_code() if k == 5 else None
    for g in MOTIF_GRAPHS:
        rows = list_motif_rows(g, k)
        hist = check_motif_rows(g, k, rows, cls5)
        assert hist == oracle.bf_motifs(g, k), (g.name, k)


def test_list_motifs_chunked_and_overflow():
    import torch

    g = gg.barabasi_albert(150, 2, seed=37)
    cls5 = _class_of_code()
    defaults = pgm.pgm_get_options()
    pgm.pgm_set_options(level_budget=1024)  # many chunks of levels 3 and 4
    try:
        for k in (3, 4, 5):
            rows = list_motif_rows(g, k)
            assert check_motif_rows(g, k, rows, cls5) == oracle.esu_motifs(g, k, threads=8), k
    finally:
        pgm.pgm_set_options(**defaults)
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        n = pgm.pgm_list_motifs(h, 4)
        buf = torch.zeros((n - 1, 5), dtype=torch.int32, device="cuda")
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_list_motifs(h, 4, buf.data_ptr(), n - 1)
        assert e.value.status == pgm.PGM_EOVERFLOW
        for bad in (2, 6):
            with pytest.raises(pgm.PgmError) as e:
                pgm.pgm_list_motifs(h, bad)
            assert e.value.status == pgm.PGM_EUNSUPPORTED
    finally:
        pgm.pgm_graph_destroy(h)


def test_list_motifs_to_host():
    """Motif rows streamed to host memory equal the device listing, also when
    the last level is cut into many staging-sized chunks."""
    g = gg.barabasi_albert(150, 2, seed=37)
    defaults = pgm.pgm_get_options()
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        for budget in (0, 1024):
            if budget:
                pgm.pgm_set_options(level_budget=budget)
            for k in (3, 4, 5):
                dev = list_motif_rows(g, k)
                n = pgm.pgm_list_motifs_host(h, k)
                out = np.full((n, k + 1), -1, np.int32)
                assert pgm.pgm_list_motifs_host(h, k, out) == n == len(dev)
                assert sorted(map(tuple, out)) == sorted(map(tuple, dev)), (budget, k)
        small = np.zeros((n - 1, 6), np.int32)
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_list_motifs_host(h, 5, small)
        assert e.value.status == pgm.PGM_EOVERFLOW
    finally:
        pgm.pgm_set_options(**defaults)
        pgm.pgm_graph_destroy(h)
