"""Parity of frequent subgraph mining (pgm_fsm, through the C ABI) with the
oracle (Sec. 2.1 FSM; Sec. 3.3 Listing 5): edge-induced embeddings of a
vertex-labelled graph, MNI support, Filter between levels.

Results are integers and pattern codes: the bar is exact equality of the
whole pattern list (canonical labels, adjacency, support, embeddings).
Families span one-warp and many-warp neighbour lists (hubs of degree far
above 32), many distinct patterns (hundreds of labels), every min_support
regime (everything frequent, nothing frequent, the Filter cutting level 1 or
2) and the degenerate graphs (no edges, one edge, disjoint parts).  At the
full workload size the oracle is too slow; there the checks are properties
that hold at any size: the embeddings of each shape sum to the graph's
closed-form totals, min_support keeps exactly the patterns at or above it,
and renumbering the vertices changes nothing.
"""
import ctypes as C

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def gpu_fsm(g, lab, max_edges, sigma=1):
    with pgm.Graph(g) as G:
        G.set_labels(lab)
        return G.fsm(max_edges, sigma)


def check(g, lab, max_edges, sigmas=(1,)):
    for s in sigmas:
        want = oracle.fsm(g, lab, max_edges, s)
        got = gpu_fsm(g, lab, max_edges, s)
        assert got == want, (g.name, max_edges, s, len(got), len(want))


# ------------------------------------------------------------ small graphs
def small_families():
    yield from (gg.complete(n) for n in (1, 2, 3, 4, 5, 9, 40))
    yield from (gg.star(s) for s in (1, 2, 3, 33, 100))
    yield from (gg.cycle(n) for n in (3, 4, 5, 37))
    yield gg.path(65)
    yield gg.empty(5)
    yield gg.from_edges(4, [(0, 1), (2, 3)])
    yield from (gg.complete_multipartite(s) for s in ((3, 3, 3), (1, 2, 3, 4), (20, 30)))


@pytest.mark.parametrize("nlab", [1, 2, 3])
def test_families(nlab):
    for i, g in enumerate(small_families()):
        lab = gg.vertex_labels(g.n, nlab, seed=7 + i)
        check(g, lab, 3, (1, 2, 5))


def test_complete_bipartite_side_labels():
    g = gg.complete_multipartite((4, 6))
    lab = np.array([0] * 4 + [1] * 6, np.int32)
    check(g, lab, 3, (1, 4, 5))


@pytest.mark.parametrize("max_edges", [1, 2, 3])
def test_random_small(max_edges):
    rng = np.random.default_rng(max_edges)
    for i in range(120):
        n = int(rng.integers(1, 31))
        g = gg.erdos_renyi(n, float(rng.uniform(0.05, 0.6)), seed=500 + i)
        lab = gg.vertex_labels(n, int(rng.integers(1, 5)), seed=900 + i)
        check(g, lab, max_edges, (1, 2, 4))


@pytest.mark.parametrize("order", [1, 2])
def test_domain_orders(order):
    """Both enumerations of the 2-edge domain passes (by first edge, by
    centre vertex in label order; the automatic choice takes the centre
    order only for bitmaps larger than half of L2) give the oracle's lists,
    with and without the Filter dropping edges."""
    try:
        pgm.pgm_set_options(fsm_domain_order=order)
        for i, g in enumerate([gg.complete(9), gg.star(40), gg.barabasi_albert(800, 3, seed=7),
                               gg.erdos_renyi(600, 0.02, seed=8), gg.empty(4)]):
            lab = gg.vertex_labels(g.n, 3, seed=20 + i, skew=0.9)
            check(g, lab, 3, (1, 3, 40))
    finally:
        pgm.pgm_set_options(fsm_domain_order=0)


# ----------------------------------------------------------- medium graphs
@pytest.mark.parametrize("sigma", [1, 20, 100, 10**6])
def test_er_medium(sigma):
    g = gg.erdos_renyi(2000, 0.005, seed=3)
    check(g, gg.vertex_labels(g.n, 6, seed=3), 3, (sigma,))


def test_hubs_skewed_labels():
    """Barabasi-Albert hubs (neighbour lists of hundreds: many 32-lane
    batches per list) with skewed labels; min_support values that make the
    Filter drop level-1 and level-2 patterns."""
    g = gg.barabasi_albert(1500, 3, seed=2)
    check(g, gg.vertex_labels(g.n, 5, seed=2, skew=1.2), 3, (1, 30, 150, 400))


@pytest.mark.parametrize("nlab,max_edges", [(100, 2), (12, 3)])
def test_many_labels(nlab, max_edges):
    """Many labels: tens of thousands of distinct patterns per level (within
    the oracle's table of 2^17 patterns)."""
    g = gg.erdos_renyi(3000, 0.003, seed=4)
    check(g, gg.vertex_labels(g.n, nlab, seed=4), max_edges, (1, 2))


@pytest.mark.parametrize("max_edges", [1, 2])
def test_rmat_levels(max_edges):
    g = gg.rmat(1 << 12, 1 << 15, seed=4)
    check(g, gg.vertex_labels(g.n, 8, seed=5, skew=0.8), max_edges, (1, 50))


def test_largest_label():
    """Labels up to 2^15 - 1 (the key's field width): K_5 and a wedge-rich
    graph with labels {0, 32767} give the patterns of labels {0, 1} with the
    label values swapped in (both sort the same way)."""
    for g in (gg.complete(5), gg.erdos_renyi(60, 0.2, seed=8)):
        lab01 = gg.vertex_labels(g.n, 2, seed=1)
        big = np.where(lab01 == 1, 32767, 0).astype(np.int32)
        want = [dict(p, labels=tuple(32767 if x == 1 else 0 for x in p["labels"]))
                for p in oracle.fsm(g, lab01, 3, 1)]
        assert gpu_fsm(g, big, 3, 1) == want


def test_repeated_calls_and_relabelling():
    """One handle, several calls (tables reused), labels replaced between them."""
    g = gg.erdos_renyi(500, 0.02, seed=6)
    l1, l2 = gg.vertex_labels(g.n, 3, seed=1), gg.vertex_labels(g.n, 4, seed=2)
    with pgm.Graph(g) as G:
        G.set_labels(l1)
        a = G.fsm(3, 5)
        b = G.fsm(2, 5)
        G.set_labels(l2)
        c = G.fsm(3, 5)
    assert a == oracle.fsm(g, l1, 3, 5)
    assert b == [p for p in a if p["edges"] <= 2]
    assert c == oracle.fsm(g, l2, 3, 5)


# -------------------------------------------------------------- the ABI
def test_errors_and_size_query():
    g = gg.erdos_renyi(200, 0.05, seed=9)
    lab = gg.vertex_labels(g.n, 3, seed=9)
    L = pgm.load()
    with pgm.Graph(g) as G:
        n = C.c_int32(-1)
        assert L.pgm_fsm(G.h, 3, 1, None, 0, C.byref(n)) == pgm.PGM_EINVAL  # no labels yet
        bad = lab.copy()
        bad[7] = 1 << 15
        with pytest.raises(pgm.PgmError):
            G.set_labels(bad)
        bad[7] = -1
        with pytest.raises(pgm.PgmError):
            G.set_labels(bad)
        G.set_labels(lab)
        assert L.pgm_fsm(G.h, 0, 1, None, 0, C.byref(n)) == pgm.PGM_EUNSUPPORTED
        assert L.pgm_fsm(G.h, 4, 1, None, 0, C.byref(n)) == pgm.PGM_EUNSUPPORTED
        assert L.pgm_fsm(G.h, 3, 0, None, 0, C.byref(n)) == pgm.PGM_EINVAL
        assert L.pgm_fsm(G.h, 3, 1, None, 0, C.byref(n)) == pgm.PGM_OK  # size query
        want = oracle.fsm(g, lab, 3, 1)
        assert n.value == len(want)
        buf = (pgm.pgm_fsm_pattern * n.value)()
        m = C.c_int32(-1)
        assert L.pgm_fsm(G.h, 3, 1, buf, n.value - 1, C.byref(m)) == pgm.PGM_EOVERFLOW
        assert m.value == n.value and buf[0].edges == 0  # nothing written
        assert L.pgm_fsm(G.h, 3, 1, buf, n.value, C.byref(m)) == pgm.PGM_OK
        assert [(p.edges, p.nv, tuple(p.labels[:p.nv]), p.adj, p.support, p.embeddings) for p in buf] == \
            [(p["edges"], len(p["labels"]), p["labels"], p["adj"], p["support"], p["embeddings"]) for p in want]


def test_table_overflow_is_an_error():
    """More distinct 2-edge patterns than the table holds: a clean
    PGM_ENOMEM with a message, and the handle stays usable."""
    g = gg.erdos_renyi(40000, 30.0 / 39999, seed=10)
    lab = gg.vertex_labels(g.n, 1 << 15, seed=10)
    with pgm.Graph(g) as G:
        G.set_labels(lab)
        with pytest.raises(pgm.PgmError) as e:
            G.fsm(2, 1)
        assert "full" in str(e.value)
        small = gg.vertex_labels(g.n, 2, seed=11)
        G.set_labels(small)
        r = G.fsm(1, 1)
    assert r == oracle.fsm(g, small, 1, 1)


# ------------------------------------------------- full workload, properties
def shape_totals(g):
    """Edge-induced embeddings of each shape, from the degrees and the
    triangle count: edges m; 2-edge paths sum C(d, 2); 3-stars sum C(d, 3);
    triangles trace(A^3) / 6; 3-paths sum over edges (d_u - 1)(d_v - 1)
    minus 3 per triangle."""
    import scipy.sparse as sp

    rp, col = np.asarray(g.rowptr), np.asarray(g.col)
    d = np.diff(rp).astype(np.int64)
    A = sp.csr_matrix((np.ones(col.size, np.int64), col, rp), shape=(g.n, g.n))
    tri = int((A @ A).multiply(A).sum()) // 6
    src = np.repeat(np.arange(g.n), d)
    paths = int(((d[src] - 1) * (d[col] - 1)).sum()) // 2 - 3 * tri
    return {(1, 2): g.m, (2, 3): int((d * (d - 1) // 2).sum()), (3, 3): tri,
            (3, 4): int((d * (d - 1) * (d - 2) // 6).sum()) + paths}


def shape_sums(res):
    out = {}
    for p in res:
        key = (p["edges"], len(p["labels"]))
        out[key] = out.get(key, 0) + p["embeddings"]
    return out


def test_mico_like_3fsm_properties():
    """The 3-FSM workload (patterns of up to 2 edges) on the Mico stand-in,
    29 skewed labels: with min_support 1 every embedding is counted once;
    higher min_support keeps exactly the patterns at or above it."""
    g = gg.mico_like()
    lab = gg.vertex_labels(g.n, 29, seed=1, skew=1.0)
    with pgm.Graph(g) as G:
        G.set_labels(lab)
        full = G.fsm(2, 1)
        want = shape_totals(g)
        assert shape_sums(full) == {k: v for k, v in want.items() if k[0] <= 2}
        for sigma in (300, 1000, 5000):
            assert G.fsm(2, sigma) == [p for p in full if p["support"] >= sigma]


def test_4fsm_properties_and_renumbering():
    """Patterns of up to 3 edges on a graph with hubs: shape totals, and the
    same result after a random renumbering of the vertices."""
    g = gg.barabasi_albert(20000, 3, seed=5)
    lab = gg.vertex_labels(g.n, 6, seed=5, skew=0.7)
    full = gpu_fsm(g, lab, 3, 1)
    assert shape_sums(full) == shape_totals(g)
    perm = np.random.default_rng(3).permutation(g.n)
    lab2 = np.empty_like(lab)
    lab2[perm] = lab
    assert gpu_fsm(gg.relabel(g, perm), lab2, 3, 1) == full
    assert gpu_fsm(g, lab, 3, 200) == [p for p in full if p["support"] >= 200]
