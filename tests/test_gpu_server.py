"""Serving: queries admitted by predicted memory, overlapping on the GPU,
return the same counts alone and in the mix."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu


def graphs():
    return [gg.barabasi_albert(3000, 6, seed=1), gg.rmat(1 << 13, 60000, seed=2), gg.erdos_renyi(2000, 0.01, seed=3),
            gg.complete(30), gg.barabasi_albert(800, 10, seed=4), gg.rmat(1 << 12, 20000, seed=5)]


def alone(g, kind, k):
    with pgm.Graph(g) as G:
        if kind == pgm.PGM_Q_MOTIF:
            return G.motifs(k)
        return [G.kcliques(3 if kind == pgm.PGM_Q_TRIANGLE else k)]


def test_mixed_stream_equals_alone_and_oracle():
    gs = graphs()
    s = pgm.pgm_server_create(8 << 30, 4)
    try:
        ids = [pgm.pgm_server_add_graph(s, g.n, g.rowptr, g.col) for g in gs]
        rng = np.random.default_rng(7)
        qs = []
        for _ in range(60):
            kind = int(rng.integers(0, 3))
            k = 4 if kind == pgm.PGM_Q_KCLIQUE else (int(rng.integers(3, 5)) if kind == pgm.PGM_Q_MOTIF else 3)
            gi = int(rng.integers(0, len(gs)))
            qs.append((kind, k, gi, pgm.pgm_server_submit(s, kind, k, ids[gi])))
        pgm.pgm_server_drain(s, 300.0)
        cache = {}
        for kind, k, gi, t in qs:
            r = pgm.pgm_server_poll(s, t)
            assert r.done == 1 and r.status == pgm.PGM_OK
            assert r.submit_s <= r.start_s <= r.finish_s
            key = (kind, k, gi)
            if key not in cache:
                cache[key] = alone(gs[gi], kind, k)
                g = gs[gi]
                ref = oracle.formula_motifs(g, k) if kind == pgm.PGM_Q_MOTIF else [
                    oracle.clique_count(g, 3 if kind == pgm.PGM_Q_TRIANGLE else k, "degree")]
                assert cache[key] == ref
            n = len(cache[key])
            assert [int(x) for x in r.counts[:n]] == cache[key]
    finally:
        pgm.pgm_server_destroy(s)


def test_admission_budget():
    g = gg.barabasi_albert(3000, 6, seed=1)
    s = pgm.pgm_server_create(1 << 16, 2)  # 64 KiB: motif-4 queries predict more
    try:
        gid = pgm.pgm_server_add_graph(s, g.n, g.rowptr, g.col)
        t_big = pgm.pgm_server_submit(s, pgm.PGM_Q_MOTIF, 4, gid)
        t_small = pgm.pgm_server_submit(s, pgm.PGM_Q_TRIANGLE, 3, gid)
        pgm.pgm_server_drain(s, 60.0)
        rb = pgm.pgm_server_poll(s, t_big)
        rs = pgm.pgm_server_poll(s, t_small)
        assert rb.done == 1 and rb.status == pgm.PGM_ENOMEM and rb.mem_bytes > (1 << 16)
        assert rs.status == pgm.PGM_OK and int(rs.counts[0]) == oracle.clique_count(g, 3, "degree")
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_server_submit(s, pgm.PGM_Q_MOTIF, 5, gid)
        assert e.value.status == pgm.PGM_EUNSUPPORTED
        with pytest.raises(pgm.PgmError):
            pgm.pgm_server_submit(s, pgm.PGM_Q_MOTIF, 3, 99)
    finally:
        pgm.pgm_server_destroy(s)


def test_drain_timeout_and_cancel():
    g = gg.rmat(1 << 14, 150000, seed=9)
    s = pgm.pgm_server_create(8 << 30, 1)
    try:
        gid = pgm.pgm_server_add_graph(s, g.n, g.rowptr, g.col)
        ts = [pgm.pgm_server_submit(s, pgm.PGM_Q_MOTIF, 4, gid) for _ in range(20)]
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_server_drain(s, 0.0)
        assert e.value.status == pgm.PGM_ETIMEOUT
    finally:
        pgm.pgm_server_destroy(s)  # cancels what is still queued, joins the workers
