"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts are integers: the bar is bit-exact equality.  Graph families span
several tiles (32-entry batches, staged segments, hub parents handled by the
block kernels) and ragged tails; options that shrink the staging capacity
and the level budget force the hub kernels, the global-memory fallbacks and
edge-blocking chunks on small inputs.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1911_06969_b300 import pgm

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
DEFAULTS = {}


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    DEFAULTS.update(pgm.pgm_get_options())
    yield
    pgm.pgm_set_options(**DEFAULTS)


@pytest.fixture
def small_tiles():
    """Tiny staging capacity and level budget: hub kernels + chunking on small graphs."""
    pgm.pgm_set_options(warp_stage_cap=32, hub_threshold=32, level_budget=1024)
    yield
    pgm.pgm_set_options(**DEFAULTS)


def gpu_cliques(g, ks):
    with pgm.Graph(g) as G:
        return [G.kcliques(k) for k in ks]


def gpu_motifs(g, k):
    with pgm.Graph(g) as G:
        return G.motifs(k)


def families():
    yield from (gg.complete(n) for n in (1, 2, 3, 5, 9, 40, 70))
    yield from (gg.complete_multipartite(s) for s in ((3, 3, 3), (1, 2, 3, 4), (8, 8, 8, 8), (20, 30)))
    yield from (gg.star(s) for s in (1, 3, 33, 100))
    yield gg.cycle(4)
    yield gg.cycle(37)
    yield gg.path(65)
    yield gg.empty(5)
    yield gg.from_edges(4, [(0, 1), (2, 3)])
    for i in range(25):
        yield gg.erdos_renyi(12 + i, 0.1 + 0.03 * i, seed=500 + i)
    yield gg.barabasi_albert(400, 6, seed=3)
    yield gg.erdos_renyi(300, 0.2, seed=4)
    yield gg.rmat(1 << 11, 12000, seed=5)


FAMILIES = list(families())


@pytest.mark.parametrize("g", FAMILIES, ids=[f"{g.name}" for g in FAMILIES])
def test_cliques_families(g):
    ks = [1, 2, 3, 4, 5, 6]
    want = [oracle.clique_count(g, k, "degree") for k in ks]
    assert gpu_cliques(g, ks) == want


@pytest.mark.parametrize("g", FAMILIES, ids=[f"{g.name}" for g in FAMILIES])
def test_motifs_families(g):
    for k in (3, 4):
        assert gpu_motifs(g, k) == oracle.formula_motifs(g, k), k


@pytest.mark.parametrize("engine", [1, 2])
def test_clique_engines(engine):
    """Level lists (1) and bitset levels (2) give the same exact counts, including
    big out-lists (block kernel) and out-lists above 512 (rows in global scratch)."""
    import itertools
    import math

    pgm.pgm_set_options(clique_engine=engine)
    try:
        for g in [gg.barabasi_albert(3000, 9, seed=41), gg.rmat(1 << 12, 40000, seed=42),
                  gg.erdos_renyi(500, 0.3, seed=43)]:
            assert gpu_cliques(g, [3, 4, 5]) == [oracle.clique_count(g, k, "degree") for k in (3, 4, 5)], g.name
        for n in (70, 600):
            assert gpu_cliques(gg.complete(n), [3, 4, 5]) == [math.comb(n, k) for k in (3, 4, 5)]
        sizes = (180, 180, 180, 180)
        want = [sum(math.prod(c) for c in itertools.combinations(sizes, k)) for k in (3, 4, 5)]
        assert gpu_cliques(gg.complete_multipartite(sizes), [3, 4, 5]) == want
    finally:
        pgm.pgm_set_options(clique_engine=0)


@pytest.mark.parametrize("engine", [1, 2])
def test_warp_grab_sizes(engine):
    """Vertex counts that set the warp kernels' grab (parents per queue
    access) anywhere from one to the full grab: a few thousand vertices (one
    per grab) up to 10^5 (the full grab), with hub vertices so that the
    bucket lists and block kernels take part too."""
    pgm.pgm_set_options(clique_engine=engine)
    try:
        for g in [gg.barabasi_albert(2000, 8, seed=61), gg.rmat(20000, 160000, seed=62),
                  gg.rmat(40000, 320000, seed=63), gg.rmat(100000, 800000, seed=64)]:
            if g.name not in _GRAB_WANT:
                _GRAB_WANT[g.name] = [oracle.clique_count(g, k, "degree") for k in (3, 4)]
            assert gpu_cliques(g, [3, 4]) == _GRAB_WANT[g.name], g.name
    finally:
        pgm.pgm_set_options(clique_engine=0)


_GRAB_WANT = {}  # oracle counts, shared by the two engines' runs


@pytest.mark.parametrize("smem_degree,fwd", [(64, 1), (256, 1000), (512, 8), (1024, 1), (1024, 1000)])
def test_bitset_buckets(smem_degree, fwd):
    """Bitset engine: every out-degree bucket (rows in shared memory up to
    bitset_smem_degree, global rows above it) and both row-building directions
    give the exact counts."""
    import itertools
    import math

    pgm.pgm_set_options(clique_engine=2, bitset_smem_degree=smem_degree, bitset_forward_ratio=fwd)
    try:
        for g in [gg.barabasi_albert(3000, 9, seed=41), gg.rmat(1 << 12, 40000, seed=42)]:
            assert gpu_cliques(g, [3, 4, 5]) == [oracle.clique_count(g, k, "degree") for k in (3, 4, 5)], g.name
        sizes = (90,) * 6  # out-degrees up to 450
        want = [sum(math.prod(c) for c in itertools.combinations(sizes, k)) for k in (3, 4, 5)]
        assert gpu_cliques(gg.complete_multipartite(sizes), [3, 4, 5]) == want
        sizes = (260,) * 5  # out-degrees up to 1040: above the largest shared-memory bucket
        want = [sum(math.prod(c) for c in itertools.combinations(sizes, k)) for k in (3, 4)]
        assert gpu_cliques(gg.complete_multipartite(sizes), [3, 4]) == want
        assert gpu_cliques(gg.complete(1100), [3, 4]) == [math.comb(1100, k) for k in (3, 4)]
    finally:
        pgm.pgm_set_options(clique_engine=0, bitset_smem_degree=1024, bitset_forward_ratio=4)


@pytest.mark.parametrize("order", [0, 1])
def test_motif_orders(order):
    """Motif counts on the degree-relabelled copy (order 0) and on the input IDs
    (order 1) both equal the oracle's, for graphs with hubs of both kinds of ID."""
    pgm.pgm_set_options(motif_order=order)
    try:
        for g in [gg.barabasi_albert(3000, 7, seed=21), gg.rmat(1 << 12, 30000, seed=22),
                  gg.chung_lu(4096, 2.1, 10.0, 500.0, 23), gg.star(50), gg.complete_multipartite((9, 10, 11))]:
            for k in (3, 4):
                assert gpu_motifs(g, k) == oracle.formula_motifs(g, k), (g.name, k, order)
    finally:
        pgm.pgm_set_options(motif_order=0)


@pytest.mark.parametrize("bmin", [1, 2, 8, 33, 1 << 30])
def test_motif_b_side_threshold(bmin):
    """4-motif counts equal the oracle's whichever level-2 edges the B-side
    kernel counts whole (f2 = 0 children >= bmin: nothing stored, closed-form
    base regions, f2 = 1 children from the scans of N(w)) and which the
    level-3 list keeps (1 = every edge from B's side, 2^30 = none), on both
    vertex orders, with hubs (bitmaps) and without, and across edge-blocking
    chunks (small level budget)."""
    try:
        for order in (0, 1):
            pgm.pgm_set_options(motif_b_side_min=bmin, motif_order=order, level_budget=4096)
            for g in [gg.barabasi_albert(2500, 9, seed=31), gg.erdos_renyi(300, 0.2, seed=32),
                      gg.chung_lu(3000, 2.1, 12.0, 600.0, 33), gg.complete(45), gg.star(70),
                      gg.complete_multipartite((12, 20, 25)), gg.cycle(50)]:
                assert gpu_motifs(g, 4) == oracle.formula_motifs(g, 4), (g.name, bmin, order)
    finally:
        pgm.pgm_set_options(motif_b_side_min=8, motif_order=0, level_budget=1 << 31)


def test_small_tiles_hub_paths(small_tiles):
    for g in [gg.barabasi_albert(2000, 12, seed=8), gg.complete(80), gg.rmat(1 << 12, 30000, seed=9),
              gg.complete_multipartite((30, 30, 30))]:
        assert gpu_cliques(g, [3, 4, 5]) == [oracle.clique_count(g, k, "degree") for k in (3, 4, 5)], g.name
        for k in (3, 4):
            assert gpu_motifs(g, k) == oracle.formula_motifs(g, k), (g.name, k)


def test_chunking_reported(small_tiles):
    # the level-list engine materialises level 3 in budget-bounded chunks
    pgm.pgm_set_options(warp_stage_cap=32, hub_threshold=32, level_budget=1024, profile=1, clique_engine=1)
    g = gg.barabasi_albert(3000, 10, seed=11)
    with pgm.Graph(g) as G:
        c4 = G.kcliques(4)
        prof = pgm.pgm_last_profile()
        m4 = G.motifs(4)
        prof4 = pgm.pgm_last_profile()
    assert c4 == oracle.clique_count(g, 4, "degree")
    assert m4 == oracle.formula_motifs(g, 4)
    assert prof["chunks"] > 1 and prof4["chunks"] > 1
    lv = oracle.clique_levels(g, 4, "degree")
    assert prof["level_size"][2:5] == lv[2:5]


def test_triangle_er4096_golden():
    d = json.load(open(os.path.join(GOLD, "triangle_er.json")))
    g = gg.triangle_er()
    lv = d["clique_levels_k7"]
    assert gpu_cliques(g, [3, 4, 5]) == lv[3:6]
    assert gpu_motifs(g, 3) == d["motif3"]
    assert gpu_motifs(g, 4) == d["motif4"]


@pytest.mark.parametrize("engine", [1, 2])
def test_level_sizes_match_oracle(engine):
    pgm.pgm_set_options(profile=1, clique_engine=engine)
    try:
        g = gg.barabasi_albert(5000, 8, seed=12)
        lv = oracle.clique_levels(g, 5, "degree")
        with pgm.Graph(g) as G:
            assert G.kcliques(5) == lv[5]
            prof = pgm.pgm_last_profile()
            assert prof["level_size"][2:6] == lv[2:6]
            assert G.kcliques(4) == lv[4]
            assert pgm.pgm_last_profile()["level_size"][2:5] == lv[2:5]
            w, t = G.motifs(3)
            prof3 = pgm.pgm_last_profile()
            m4 = G.motifs(4)
            prof4 = pgm.pgm_last_profile()
        assert prof3["level_size"][3] == w + t
        assert prof4["level_size"][3] == w + t  # |L3| = connected 3-sets
        assert prof4["level_size"][4] == sum(m4)
    finally:
        pgm.pgm_set_options(profile=0, clique_engine=0)


def test_range_additivity():
    g = gg.barabasi_albert(3000, 7, seed=13)
    cuts = [0, 1, 700, 701, 1500, 2999, 3000]
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        for k in (3, 4):
            parts = [pgm.pgm_count_kcliques_range(h, k, a, b) for a, b in zip(cuts, cuts[1:])]
            assert sum(parts) == pgm.pgm_count_kcliques(h, k)
        for k in (3, 4):
            parts = np.array([pgm.pgm_count_motifs_range(h, k, a, b) for a, b in zip(cuts, cuts[1:])],
                             dtype=object)
            assert list(parts.sum(0)) == pgm.pgm_count_motifs(h, k)
            # the oracle's ESU roots are the minimum vertex of each set, as on the GPU
            assert [int(x) for x in parts[2]] == oracle.esu_motifs(g, k, roots=(cuts[2], cuts[3]))
    finally:
        pgm.pgm_graph_destroy(h)


def test_relabel_invariance():
    g = gg.rmat(1 << 12, 25000, seed=14)
    h = gg.relabel(g, np.random.default_rng(3).permutation(g.n))
    assert gpu_cliques(g, [3, 4, 5]) == gpu_cliques(h, [3, 4, 5])
    assert gpu_motifs(g, 4) == gpu_motifs(h, 4)


def test_orientation_stats():
    g = gg.rmat(1 << 12, 25000, seed=15)
    deg = np.diff(g.rowptr)
    src = np.repeat(np.arange(g.n), deg)
    keep = (deg[src] < deg[g.col]) | ((deg[src] == deg[g.col]) & (src < g.col))
    outdeg = np.bincount(src[keep], minlength=g.n)
    with pgm.Graph(g) as G:
        G.orient()
        st = G.stats()
    s2, s3, dmax = oracle.degree_sums(g)
    assert st["m"] == g.m and st["n"] == g.n and st["dmax"] == dmax
    assert st["dag_dmax"] == outdeg.max() and keep.sum() == g.m
    assert st["sum_c2"] == s2 and st["sum_c3"] == s3


def test_scan_worked_example_and_ragged():
    import torch

    d = json.load(open(os.path.join(GOLD, "inspection_execution.json")))
    for counts in [d["counts"], [], [5], list(np.random.default_rng(1).integers(0, 1000, 4095)),
                   list(np.random.default_rng(2).integers(0, 70000, 4097)),
                   list(np.random.default_rng(3).integers(0, 3, 1_000_003))]:
        c = torch.tensor(np.asarray(counts, dtype=np.int64).astype(np.int32), device="cuda")
        out = torch.empty(len(counts) + 1, dtype=torch.int64, device="cuda")
        pgm.pgm_exclusive_scan_dev(c.data_ptr() if len(counts) else 0, len(counts), out.data_ptr())
        want = oracle.exclusive_scan(counts)
        assert np.array_equal(out.cpu().numpy(), want)
        if counts == d["counts"]:
            assert list(want[:-1]) == d["start"] and want[-1] == d["total"]


def test_validation_and_sanitize():
    good = gg.erdos_renyi(50, 0.2, seed=16)
    bad = {
        "self-loop": gg.CSR(3, np.array([0, 2, 3, 4]), np.array([0, 1, 0, 0], np.int32)),
        "asymmetric": gg.CSR(3, np.array([0, 1, 1, 1]), np.array([1], np.int32)),
        "unsorted": gg.CSR(3, np.array([0, 2, 3, 4]), np.array([2, 1, 0, 0], np.int32)),
        "duplicate": gg.CSR(2, np.array([0, 2, 4]), np.array([1, 1, 0, 0], np.int32)),
        "range": gg.CSR(2, np.array([0, 1, 2]), np.array([5, 0], np.int32)),
    }
    for name, g in bad.items():
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col, pgm.PGM_VALIDATE)
        assert e.value.status == pgm.PGM_EINVAL, name
    h = pgm.pgm_graph_create_csr(good.n, good.rowptr, good.col, pgm.PGM_VALIDATE)
    pgm.pgm_graph_destroy(h)
    # row pointers are checked on the device even without PGM_VALIDATE
    with pytest.raises(pgm.PgmError) as e:
        pgm.pgm_graph_create_csr(3, np.array([0, 2, 1, 2], np.int64), np.array([1, 2], np.int32))
    assert e.value.status == pgm.PGM_EINVAL and "decreases at vertex 1" in str(e.value)
    # sanitize: an asymmetric list with a loop and a duplicate becomes the simple graph
    rp = np.array([0, 3, 4, 4], np.int64)
    col = np.array([1, 1, 0, 2], np.int32)  # 0:{1,1,0} 1:{2} 2:{}
    h = pgm.pgm_graph_create_csr(3, rp, col, pgm.PGM_SANITIZE | pgm.PGM_VALIDATE)
    try:
        assert pgm.pgm_count_motifs(h, 3) == [1, 0]  # path 0-1-2
        assert pgm.pgm_graph_stats_get(h)["m"] == 2
    finally:
        pgm.pgm_graph_destroy(h)
    # an unvalidated asymmetric graph is refused at orientation, not miscounted
    g = bad["asymmetric"]
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        with pytest.raises(pgm.PgmError) as e:
            pgm.pgm_count_kcliques(h, 3)
        assert e.value.status == pgm.PGM_EINVAL
    finally:
        pgm.pgm_graph_destroy(h)


def test_bad_arguments_and_degenerate_graphs():
    g = gg.complete(5)
    h = pgm.pgm_graph_create_csr(g.n, g.rowptr, g.col)
    try:
        for k in (0, 11):
            with pytest.raises(pgm.PgmError) as e:
                pgm.pgm_count_kcliques(h, k)
            assert e.value.status == pgm.PGM_EUNSUPPORTED
        for k in (2, 6):
            with pytest.raises(pgm.PgmError) as e:
                pgm.pgm_count_motifs(h, k)
            assert e.value.status == pgm.PGM_EUNSUPPORTED
        assert pgm.pgm_count_motifs(h, 5) == [0] * 20 + [1]  # K5: one 5-clique (last class)
        with pytest.raises(pgm.PgmError):
            pgm.pgm_count_kcliques_range(h, 3, 3, 2)
        assert pgm.pgm_count_kcliques(h, 5) == 1 and pgm.pgm_count_kcliques(h, 1) == 5
        assert pgm.pgm_count_kcliques(h, 6) == 0
    finally:
        pgm.pgm_graph_destroy(h)
    h = pgm.pgm_graph_create_csr(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    try:
        assert pgm.pgm_count_kcliques(h, 4) == 0 and pgm.pgm_count_motifs(h, 4) == [0] * 6
        assert pgm.pgm_count_motifs(h, 5) == [0] * 21
    finally:
        pgm.pgm_graph_destroy(h)


def test_device_input_path():
    import torch

    g = gg.barabasi_albert(1000, 5, seed=17)
    rp = torch.tensor(g.rowptr, device="cuda")
    col = torch.tensor(g.col, device="cuda")
    h = pgm.pgm_graph_create_csr_dev(g.n, rp.data_ptr(), col.data_ptr(), g.narcs, pgm.PGM_VALIDATE)
    try:
        assert pgm.pgm_count_kcliques(h, 4) == oracle.clique_count(g, 4, "degree")
        assert pgm.pgm_count_motifs(h, 4) == oracle.formula_motifs(g, 4)
    finally:
        pgm.pgm_graph_destroy(h)


# ------------------------------------------------------------ full sizes
def test_rmat21_cliques_golden():
    d = json.load(open(os.path.join(GOLD, "rmat21.json")))
    g = gg.rmat21()
    lv = d["clique_levels_k4"]
    with pgm.Graph(g) as G:
        assert G.kcliques(3) == lv[3]
        assert G.kcliques(4) == lv[4]
        p5 = os.path.join(GOLD, "rmat21_k5.json")
        if os.path.exists(p5):
            assert G.kcliques(5) == json.load(open(p5))["clique_levels_k5"][5]


def test_chung_lu_1m_motifs_golden():
    d = json.load(open(os.path.join(GOLD, "chung_lu_1m.json")))
    g = gg.chung_lu_1m()
    with pgm.Graph(g) as G:
        assert G.motifs(3) == d["motif3"]
        assert G.motifs(4) == d["motif4"]


def _join_independent(nb, p, seed):
    """An independent set A of nb vertices joined to every vertex of an
    Erdos-Renyi graph H on nb vertices (edge probability p).  Every vertex
    of A has out-degree nb in the DAG (H's vertices have the higher degree),
    and the k-cliques are a vertex of A with a (k-1)-clique of H, or a
    k-clique of H."""
    rng = np.random.default_rng(seed)
    A, Bv = np.arange(nb), np.arange(nb, 2 * nb)
    join = np.stack(np.meshgrid(A, Bv, indexing="ij"), -1).reshape(-1, 2)
    iu = np.triu_indices(nb, 1)
    keep = rng.random(len(iu[0])) < p
    h_edges = np.stack([iu[0][keep], iu[1][keep]], 1)
    g = gg.from_edges(2 * nb, np.concatenate([join, h_edges + nb]), f"join{nb}_p{p}")
    return g, gg.from_edges(nb, h_edges, f"H{nb}_p{p}")


@pytest.mark.parametrize("smem_degree", [1024, 256])
def test_bitset_deep(smem_degree):
    """k = 6..10 on the bitset engine (the depth-first walk over bit rows):
    every out-degree bucket, rows in shared and in global memory, exact
    counts and per-level sizes against the oracle, closed forms, and the
    level-list engine on the same graph."""
    import itertools
    import math

    saved = pgm.pgm_get_options()
    pgm.pgm_set_options(clique_engine=2, bitset_smem_degree=smem_degree)
    try:
        for g, ks in [(gg.rmat(1 << 12, 40000, seed=42), (6, 7, 8, 9)),
                      (gg.barabasi_albert(3000, 9, seed=41), (6, 7, 8, 9, 10))]:
            assert gpu_cliques(g, ks) == [oracle.clique_count(g, k, "degree", threads=8) for k in ks], g.name
        assert gpu_cliques(gg.complete(40), range(6, 11)) == [math.comb(40, k) for k in range(6, 11)]
        sizes = (12,) * 9  # out-degrees up to 96
        want = [sum(math.prod(c) for c in itertools.combinations(sizes, k)) for k in (6, 7, 8)]
        assert gpu_cliques(gg.complete_multipartite(sizes), [6, 7, 8]) == want
        # out-degrees 200 / 400 / 900 / 1100: the 256, 512, 1024 and global-row buckets
        for nb, p in [(200, 0.3), (400, 0.2), (900, 0.12), (1100, 0.1)]:
            g, h = _join_independent(nb, p, seed=nb)
            hc = [oracle.clique_count(h, k, "id", threads=8) for k in (5, 6, 7)]
            assert gpu_cliques(g, [6, 7]) == [nb * hc[0] + hc[1], nb * hc[1] + hc[2]], g.name
        # per-level sizes of one count
        g = gg.rmat(1 << 12, 40000, seed=42)
        pgm.pgm_set_options(clique_engine=2, bitset_smem_degree=smem_degree, profile=1)
        with pgm.Graph(g) as G:
            G.kcliques(8)
            sizes = pgm.pgm_last_profile()["level_size"]
        assert sizes[1:9] == oracle.clique_levels(g, 8, "degree", threads=8)[1:9]
    finally:
        pgm.pgm_set_options(**saved)
    pgm.pgm_set_options(clique_engine=1)
    try:
        g = gg.rmat(1 << 12, 40000, seed=42)
        assert gpu_cliques(g, [6, 7]) == [oracle.clique_count(g, k, "degree", threads=8) for k in (6, 7)]
    finally:
        pgm.pgm_set_options(**saved)


@pytest.mark.parametrize("engine", [1, 2])
def test_count_overflow_status(engine):
    """PGM_EOVERFLOW: with the accumulators started 2^x below 2^64
    (options.count_headroom_log2 = x), a count below 2^x comes back exact
    and a count of 2^x or more fails with PGM_EOVERFLOW -- for clique counts
    on both engines and for motif counts (k = 3, 4, 5), whose per-warp
    partials are signed (region corrections).  No fault is involved: the
    start value is an ordinary host write."""
    saved = pgm.pgm_get_options()
    d = json.load(open(os.path.join(GOLD, "triangle_er.json")))
    gc = gg.barabasi_albert(2000, 8, seed=17)
    g5 = gg.erdos_renyi(200, 0.05, seed=9)
    cases = [(gc, "kcliques", k, [oracle.clique_count(gc, k, "degree", threads=8)]) for k in (3, 4, 5)]
    cases += [(gg.triangle_er(), "motifs", k, d[f"motif{k}"]) for k in (3, 4)]
    cases += [(g5, "motifs", 5, oracle.esu_motifs(g5, 5))]
    try:
        for g, fn, k, want in cases:
            x = max(want).bit_length()  # the largest count is in [2^(x-1), 2^x)
            assert x >= 2, (g.name, k)
            with pgm.Graph(g) as G:
                call = (lambda: [G.kcliques(k)]) if fn == "kcliques" else (lambda: G.motifs(k))
                pgm.pgm_set_options(clique_engine=engine, count_headroom_log2=x)
                assert call() == want, (g.name, fn, k)
                pgm.pgm_set_options(clique_engine=engine, count_headroom_log2=x - 1)
                with pytest.raises(pgm.PgmError) as e:
                    call()
                assert e.value.status == pgm.PGM_EOVERFLOW, (g.name, fn, k)
                pgm.pgm_set_options(clique_engine=engine, count_headroom_log2=0)
                assert call() == want, (g.name, fn, k)
    finally:
        pgm.pgm_set_options(**saved)
