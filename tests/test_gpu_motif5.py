"""5-motif counts (21 classes, generic classification) of the CUDA path
against the oracle (brute force on small graphs, ESU on larger ones), on
the input IDs and on the degree-relabelled copy, with edge blocking."""
import functools

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu


def gpu5(g):
    with pgm.Graph(g) as G:
        return G.motifs(5)


SMALL = [gg.complete(5), gg.complete(9), gg.star(6), gg.cycle(5), gg.cycle(11), gg.path(12),
         gg.complete_multipartite((3, 4)), gg.complete_multipartite((2, 3, 4)), gg.empty(6),
         gg.from_edges(7, [(0, 1), (1, 2), (3, 4), (4, 5), (5, 6)])]
SMALL += [gg.erdos_renyi(16 + i, 0.15 + 0.04 * i, seed=700 + i) for i in range(10)]


@pytest.mark.parametrize("order", [0, 1])
def test_motif5_small_vs_brute_force(order):
    pgm.pgm_set_options(motif_order=order)
    try:
        for g in SMALL:
            assert gpu5(g) == oracle.bf_motifs(g, 5), (g.name, order)
    finally:
        pgm.pgm_set_options(motif_order=0)


LARGER = [gg.barabasi_albert(300, 3, seed=41), gg.rmat(1 << 8, 700, seed=42),
          gg.erdos_renyi(200, 0.05, seed=43), gg.chung_lu(512, 2.1, 6.0, 40.0, 44)]


@functools.lru_cache(maxsize=None)
def esu5(i):
    return oracle.esu_motifs(LARGER[i], 5, threads=8)


@pytest.mark.parametrize("order", [0, 1])
def test_motif5_larger_vs_esu(order):
    pgm.pgm_set_options(motif_order=order)
    try:
        for i, g in enumerate(LARGER):
            assert gpu5(g) == esu5(i), (g.name, order)
    finally:
        pgm.pgm_set_options(motif_order=0)


def test_motif5_chunks_and_ranges():
    g = gg.barabasi_albert(300, 4, seed=45)
    want = oracle.esu_motifs(g, 5, threads=8)
    defaults = pgm.pgm_get_options()
    pgm.pgm_set_options(level_budget=1024, profile=1)  # many chunks at levels 3 and 4
    try:
        with pgm.Graph(g) as G:
            assert G.motifs(5) == want
            assert pgm.pgm_last_profile()["chunks"] > 1
    finally:
        pgm.pgm_set_options(**defaults)
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        cuts = [0, 1, 170, 171, 260, 300]
        parts = np.array([pgm.pgm_count_motifs_range(h, 5, a, b) for a, b in zip(cuts, cuts[1:])], dtype=object)
        assert list(parts.sum(0)) == want
        assert [int(x) for x in parts[3]] == oracle.esu_motifs(g, 5, roots=(171, 260), threads=8)
        out = np.zeros(6, np.uint64)
        assert pgm.load().pgm_count_motifs(h, 5, out.ctypes.data, 6) == pgm.PGM_EINVAL
    finally:
        pgm.pgm_graph_destroy(h)
