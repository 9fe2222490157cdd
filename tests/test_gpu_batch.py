"""Batched counting of many graphs in one pass: per-graph counts equal the
oracle's, the per-graph loop's, and those of every autotuned schedule and of
CUDA-graph replays."""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def make_batch(b):
    return pgm.pgm_batch_create(b.G, b.vtx_off, b.graph.rowptr, b.graph.col, pgm.PGM_VALIDATE)


def mixed_batch():
    parts = [gg.empty(0), gg.complete(7), gg.star(40), gg.empty(3), gg.cycle(9)]
    parts += [gg.erdos_renyi(30 + 7 * i, 0.15, seed=40 + i) for i in range(12)]
    parts += [gg.barabasi_albert(200 + 50 * i, 3 + i % 5, seed=60 + i) for i in range(12)]
    parts += [gg.complete_multipartite((5, 6, 7)), gg.rmat(1 << 10, 6000, seed=70)]
    return gg.disjoint_union(parts), parts


def test_batch_motifs_and_cliques_match_oracle():
    b, parts = mixed_batch()
    h = make_batch(b)
    try:
        for k in (3, 4):
            want = oracle.formula_motifs_batch(b, k)
            got = pgm.pgm_batch_count_motifs(h, k)
            assert np.array_equal(got, want), k
            assert np.array_equal(pgm.pgm_batch_count_motifs_loop(h, k), want), k
        for k in (1, 2, 3, 4, 5):
            got = pgm.pgm_batch_count_kcliques(h, k)
            assert [int(x) for x in got] == [oracle.clique_count(p, k, "degree") for p in parts], k
    finally:
        pgm.pgm_batch_destroy(h)


def test_graph_replay_and_autotune():
    b = gg.batch_small(300, nmin=16, nmax=600, seed=5)
    h = make_batch(b)
    try:
        want = oracle.formula_motifs_batch(b, 4)
        tune, ms = pgm.pgm_batch_autotune(h, 4)
        assert tune.use_graph == 1 and ms > 0
        for _ in range(3):  # capture on the first call, replay afterwards
            assert np.array_equal(pgm.pgm_batch_count_motifs(h, 4, tune), want)
        t2 = pgm.pgm_tune(256, 64, 32, 0, 1)
        assert np.array_equal(pgm.pgm_batch_count_motifs(h, 4, t2), want)
        assert np.array_equal(pgm.pgm_batch_count_motifs(h, 4, tune), want)
        w3 = oracle.formula_motifs_batch(b, 3)
        assert np.array_equal(pgm.pgm_batch_count_motifs(h, 3, tune), w3)
        t3 = pgm.pgm_tune(0, 0, 0, 0, 1)
        k4 = pgm.pgm_batch_count_kcliques(h, 4, t3)
        assert [int(x) for x in k4] == [oracle.clique_count(b.part(i), 4, "degree") for i in range(b.G)]
    finally:
        pgm.pgm_batch_destroy(h)


def test_autotune_trials_and_cache(tmp_path):
    """pgm_batch_autotune_ex: the first call times candidates (every trial
    listed, the winner the fastest of them, counts exact under it) and
    writes the winner to a JSON cache keyed by the batch's features; the
    second call returns the same setting from the cache without timing."""
    import json

    b = gg.batch_small(200, nmin=16, nmax=400, seed=6)
    h = make_batch(b)
    cache = str(tmp_path / "tune.json")
    try:
        want = oracle.formula_motifs_batch(b, 4)
        t1, ms1, trials, hit1 = pgm.pgm_batch_autotune_ex(h, 4, cache)
        assert not hit1 and len(trials) >= 8
        assert ms1 == min(ms for _, ms in trials)
        assert t1.use_graph == 1
        assert np.array_equal(pgm.pgm_batch_count_motifs(h, 4, t1), want)
        for tt, _ in trials:  # every knob combination tried gives the same counts
            t = pgm.pgm_tune(**{k: v for k, v in tt.items() if k != "use_graph"})
            assert np.array_equal(pgm.pgm_batch_count_motifs(h, 4, t), want), tt
        t2, ms2, trials2, hit2 = pgm.pgm_batch_autotune_ex(h, 4, cache)
        assert hit2 and trials2 == [] and t2.as_dict() == t1.as_dict() and abs(ms2 - ms1) < 1e-2
        entries = json.load(open(cache))
        assert len(entries) == 1 and list(entries)[0].startswith("motif4_G2^7_")
    finally:
        pgm.pgm_batch_destroy(h)


def test_batch_rejects_crossing_arcs():
    g = gg.path(6)  # vertices 0..5; split as two graphs of 3 -> arc 2-3 crosses
    with pytest.raises(pgm.PgmError) as e:
        pgm.pgm_batch_create(2, np.array([0, 3, 6]), g.rowptr, g.col)
    assert e.value.status == pgm.PGM_EINVAL


def test_small_batch_20k_golden():
    d = json.load(open(os.path.join(GOLD, "small_batch_20k.json")))
    b = gg.small_batch_20k()
    h = make_batch(b)
    try:
        got = pgm.pgm_batch_count_motifs(h, 4, pgm.pgm_tune(0, 0, 0, 0, 1))
        assert [[int(x) for x in r] for r in got[:64]] == d["motif4_first64"]
        assert [int(x) for x in got.astype(object).sum(0)] == d["motif4_total"]
        assert hashlib.sha256(np.ascontiguousarray(got, np.uint64).tobytes()).hexdigest() == d["motif4_sha256"]
    finally:
        pgm.pgm_batch_destroy(h)


def test_batch_motifs5():
    """5-motif counts per graph of a batch (21 classes each): direct pass,
    CUDA-graph replay and the per-graph loop all equal the oracle's."""
    parts = [gg.empty(0), gg.complete(7), gg.star(12), gg.empty(2), gg.cycle(9), gg.path(8),
             gg.complete_multipartite((3, 4, 4))]
    parts += [gg.erdos_renyi(30 + 5 * i, 0.15, seed=80 + i) for i in range(6)]
    parts += [gg.barabasi_albert(80 + 20 * i, 2 + i % 3, seed=90 + i) for i in range(6)]
    b = gg.disjoint_union(parts)
    want = np.array([oracle.esu_motifs(p, 5) for p in parts], dtype=np.uint64)
    h = make_batch(b)
    try:
        assert np.array_equal(pgm.pgm_batch_count_motifs(h, 5), want)
        assert np.array_equal(pgm.pgm_batch_count_motifs_loop(h, 5), want)
        t = pgm.pgm_tune(256, 512, 512, 0, 1)
        for _ in range(2):  # capture, then replay
            assert np.array_equal(pgm.pgm_batch_count_motifs(h, 5, t), want)
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_batch_count_motifs(h, 6)
        assert e.value.status == pgm.PGM_EUNSUPPORTED
    finally:
        pgm.pgm_batch_destroy(h)
