"""Pins for the CPU oracle, checked against facts outside the oracle itself.

The oracle (``oracle/``) is pinned by: closed forms on graph families whose
clique and motif counts follow from elementary combinatorics; degree
identities; brute force over all subsets of small random graphs; invariance
under relabelling / isolated vertices / disjoint union; agreement between
independent tiers; and the paper's worked examples (``tests/golden``).
Each family below is chosen so that a dropped term, a wrong coefficient or a
transposed pattern index in the oracle fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
C = math.comb


def e_sym(sizes, k):
    """Elementary symmetric polynomial e_k(sizes): k-cliques of a complete multipartite graph."""
    return sum(math.prod(c) for c in itertools.combinations(sizes, k))


def all_tiers_motifs(g, k):
    res = {"formula": oracle.formula_motifs(g, k), "esu": oracle.esu_motifs(g, k)}
    if g.n <= 64:
        res["bf"] = oracle.bf_motifs(g, k)
    return res


def all_tiers_cliques(g, k):
    res = {"id": oracle.clique_count(g, k, "id"), "degree": oracle.clique_count(g, k, "degree")}
    if g.n <= 64 and k <= 8:
        res["bf"] = oracle.bf_cliques(g, k)
    return res


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 10])
def test_complete_graph(n):
    g = gg.complete(n)
    for k in range(1, 8):
        for name, v in all_tiers_cliques(g, k).items():
            assert v == C(n, k), (name, k)
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == [0, C(n, 3)], name
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [0, 0, 0, 0, 0, C(n, 4)], name


@pytest.mark.parametrize("sizes", [(3, 3, 3), (1, 2, 3, 4), (5, 5), (2, 2, 2, 2, 2), (4, 1, 1, 6)])
def test_complete_multipartite(sizes):
    """Turan-type graphs have many degree ties, exercising the (degree, ID) order."""
    g = gg.complete_multipartite(sizes)
    for k in range(1, 7):
        for name, v in all_tiers_cliques(g, k).items():
            assert v == e_sym(sizes, k), (name, k)


@pytest.mark.parametrize("s", [0, 1, 2, 3, 5, 9])
def test_star(s):
    g = gg.star(s)
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == [C(s, 2), 0], name
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [C(s, 3), 0, 0, 0, 0, 0], name
    for k in (3, 4):
        assert oracle.clique_count(g, k) == 0


@pytest.mark.parametrize("n", [5, 6, 9, 20])
def test_cycle(n):
    g = gg.cycle(n)
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == [n, 0], name
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [0, n, 0, 0, 0, 0], name


def test_small_cycles():
    assert oracle.bf_motifs(gg.cycle(4), 4) == [0, 0, 0, 1, 0, 0]
    assert oracle.formula_motifs(gg.cycle(4), 4) == [0, 0, 0, 1, 0, 0]
    assert oracle.esu_motifs(gg.cycle(4), 4) == [0, 0, 0, 1, 0, 0]
    assert oracle.formula_motifs(gg.cycle(3), 3) == [0, 1]


@pytest.mark.parametrize("n", [3, 4, 6, 11])
def test_path(n):
    g = gg.path(n)
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == [n - 2, 0], name
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [0, max(n - 3, 0), 0, 0, 0, 0], name


@pytest.mark.parametrize("a,b", [(2, 2), (2, 3), (3, 4), (1, 6), (5, 5)])
def test_complete_bipartite(a, b):
    g = gg.complete_multipartite((a, b))
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == [a * C(b, 2) + b * C(a, 2), 0], name
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [a * C(b, 3) + b * C(a, 3), 0, 0, C(a, 2) * C(b, 2), 0, 0], name


# One graph per 4-vertex pattern: each must land in its own class, which
# pins the classification and the output order independently of formulas.
PATTERNS4 = {
    0: [(0, 1), (0, 2), (0, 3)],  # 3-star
    1: [(0, 1), (1, 2), (2, 3)],  # 4-path
    2: [(0, 1), (1, 2), (0, 2), (2, 3)],  # tailed triangle
    3: [(0, 1), (1, 2), (2, 3), (3, 0)],  # 4-cycle
    4: [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)],  # diamond
    5: [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)],  # 4-clique
}


@pytest.mark.parametrize("p", sorted(PATTERNS4))
def test_single_pattern(p):
    g = gg.from_edges(4, PATTERNS4[p])
    want = [0] * 6
    want[p] = 1
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == want, name


def test_disconnected_sets_not_counted():
    # triangle + isolated vertex: 3 edges on 4 vertices but not connected
    g = gg.from_edges(4, [(0, 1), (1, 2), (0, 2)])
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [0] * 6, name
    # two disjoint edges: not connected
    g = gg.from_edges(4, [(0, 1), (2, 3)])
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == [0] * 6, name


# --------------------------------------------------------------- identities
def _random_graphs(count, nmax=12, seed0=100):
    rng = np.random.default_rng(1234)
    for i in range(count):
        n = int(rng.integers(1, nmax + 1))
        p = float(rng.choice([0.15, 0.3, 0.5, 0.7, 0.9]))
        yield gg.erdos_renyi(n, p, seed=seed0 + i)


def test_brute_force_agreement_small_random():
    """All tiers agree with brute force on several hundred graphs with n <= 12."""
    for g in _random_graphs(300):
        for k in (3, 4):
            bf = oracle.bf_motifs(g, k)
            assert oracle.esu_motifs(g, k) == bf, (g.name, k)
            assert oracle.formula_motifs(g, k) == bf, (g.name, k)
        for k in range(1, 7):
            bf = oracle.bf_cliques(g, k)
            assert oracle.clique_count(g, k, "id") == bf, (g.name, k)
            assert oracle.clique_count(g, k, "degree") == bf, (g.name, k)


def test_brute_force_agreement_n64():
    for i, p in enumerate([0.1, 0.2, 0.35]):
        g = gg.erdos_renyi(40, p, seed=7 + i)
        assert oracle.formula_motifs(g, 4) == oracle.bf_motifs(g, 4)
        assert oracle.esu_motifs(g, 4) == oracle.bf_motifs(g, 4)
        assert oracle.clique_count(g, 5) == oracle.bf_cliques(g, 5)


def test_degree_identities():
    """sum C(d,2) = wedges + 3 triangles; sum C(d,3) = S + T + 2D + 4K."""
    for g in list(_random_graphs(40, nmax=30)) + [gg.triangle_er(), gg.barabasi_albert(500, 4, seed=3)]:
        s2, s3, _ = oracle.degree_sums(g)
        w, t = oracle.formula_motifs(g, 3)
        assert s2 == w + 3 * t
        S, P, T, Cy, D, K = oracle.esu_motifs(g, 4)
        assert s3 == S + T + 2 * D + 4 * K
        assert oracle.clique_count(g, 3) == t


def test_relabel_and_isolated_invariance():
    g = gg.barabasi_albert(300, 5, seed=9)
    perm = np.random.default_rng(5).permutation(g.n)
    h = gg.relabel(g, perm)
    assert oracle.formula_motifs(h, 4) == oracle.formula_motifs(g, 4)
    assert oracle.esu_motifs(h, 4) == oracle.esu_motifs(g, 4)
    for k in (3, 4, 5):
        assert oracle.clique_count(h, k, "id") == oracle.clique_count(g, k, "degree")
    # isolated vertices change nothing
    e = np.stack([np.repeat(np.arange(g.n), np.diff(g.rowptr)), g.col], 1)
    big = gg.from_edges(g.n + 50, e)
    assert oracle.formula_motifs(big, 4) == oracle.formula_motifs(g, 4)


def test_disjoint_union_additivity():
    parts = [gg.erdos_renyi(60, 0.2, seed=s) for s in range(4)] + [gg.complete(6), gg.star(7)]
    b = gg.disjoint_union(parts)
    per = oracle.formula_motifs_batch(b, 4)
    for i, p in enumerate(parts):
        assert list(per[i]) == oracle.esu_motifs(p, 4)
    assert [int(x) for x in per.sum(0)] == oracle.formula_motifs(b.graph, 4)


def test_roots_partition_sums():
    """Per-root-range clique levels add up to the whole (sharding basis)."""
    g = gg.triangle_er()
    whole = oracle.clique_levels(g, 5)
    parts = [oracle.clique_levels(g, 5, roots=(lo, min(lo + 1000, g.n))) for lo in range(0, g.n, 1000)]
    assert [sum(p[l] for p in parts) for l in range(6)] == whole
    assert whole[1] == g.n and whole[2] == g.m


def test_tiers_agree_er4096():
    g = gg.triangle_er()
    f = oracle.formula_motifs(g, 4)
    assert oracle.esu_motifs(g, 4) == f
    assert oracle.formula_motifs(g, 3) == oracle.esu_motifs(g, 3)
    for k in (3, 4, 5):
        assert oracle.clique_count(g, k, "id") == oracle.clique_count(g, k, "degree")


# ------------------------------------------------------- worked examples
def test_inspection_execution_example():
    d = json.load(open(os.path.join(GOLD, "inspection_execution.json")))
    out = oracle.exclusive_scan(d["counts"])
    assert list(out[:-1]) == d["start"] and out[-1] == d["total"]


def test_binary_search_example():
    d = json.load(open(os.path.join(GOLD, "binary_search_example.json")))
    g = gg.from_edges(d["n"], d["edges"])
    mask = oracle.connectivity_mask(g, d["embedding"], d["candidate"])
    assert [bool(mask >> j & 1) for j in range(3)] == d["connected"]


def test_automorphism_example():
    d = json.load(open(os.path.join(GOLD, "automorphism_example.json")))
    g = gg.from_edges(d["n"], d["edges"])
    for name, v in all_tiers_motifs(g, 4).items():
        assert v == d["motif4"], name
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == d["motif3"], name


def test_reduce_example():
    d = json.load(open(os.path.join(GOLD, "reduce_example.json")))
    g = gg.from_edges(d["n"], d["edges"])
    for name, v in all_tiers_motifs(g, 3).items():
        assert v == [d["motif3"]["wedge"], d["motif3"]["triangle"]], name


# ------------------------------------------------ planted-mistake checks
def _pin_suite_passes() -> bool:
    """Run a compact version of the pins above; True iff all hold."""
    try:
        for n in (4, 5, 7):
            g = gg.complete(n)
            if oracle.formula_motifs(g, 4) != [0, 0, 0, 0, 0, C(n, 4)]:
                return False
            if oracle.esu_motifs(g, 3) != [0, C(n, 3)]:
                return False
            if [oracle.clique_count(g, k, o) for k in (3, 4) for o in ("id", "degree")] != [
                    C(n, 3), C(n, 3), C(n, 4), C(n, 4)]:
                return False
        for sizes in ((2, 3), (3, 3, 3), (1, 2, 3, 4)):
            g = gg.complete_multipartite(sizes)
            if [oracle.clique_count(g, k, "degree") for k in (3, 4)] != [e_sym(sizes, 3), e_sym(sizes, 4)]:
                return False
        a, b = 3, 4
        g = gg.complete_multipartite((a, b))
        want = [a * C(b, 3) + b * C(a, 3), 0, 0, C(a, 2) * C(b, 2), 0, 0]
        if oracle.formula_motifs(g, 4) != want or oracle.esu_motifs(g, 4) != want:
            return False
        for p, e in PATTERNS4.items():
            w = [0] * 6
            w[p] = 1
            g = gg.from_edges(4, e)
            if oracle.formula_motifs(g, 4) != w or oracle.esu_motifs(g, 4) != w or oracle.bf_motifs(g, 4) != w:
                return False
        for n in (5, 8):
            if oracle.formula_motifs(gg.cycle(n), 4) != [0, n, 0, 0, 0, 0]:
                return False
            if oracle.formula_motifs(gg.path(n), 3) != [n - 2, 0]:
                return False
        if oracle.formula_motifs(gg.star(6), 4) != [C(6, 3), 0, 0, 0, 0, 0]:
            return False
        for g in _random_graphs(60, nmax=10):
            s2, s3, _ = oracle.degree_sums(g)
            w, t = oracle.formula_motifs(g, 3)
            S, P, T, Cy, D, K = oracle.formula_motifs(g, 4)
            if s2 != w + 3 * t or s3 != S + T + 2 * D + 4 * K:
                return False
            if oracle.bf_motifs(g, 4) != [S, P, T, Cy, D, K]:
                return False
    except RuntimeError:
        return False
    return True


MUTATIONS = [
    ("diamond coefficient", "i128 D = Dp - 6 * K;", "i128 D = Dp - 5 * K;"),
    ("cycle-from-diamond term dropped", "i128 C = Cp - D - 3 * K;", "i128 C = Cp - 3 * K;"),
    ("path triangle correction", "Pp -= 3 * T3;", "Pp -= 2 * T3;"),
    ("tailed-triangle vs 4-cycle swapped", "case 4: return maxdeg == 3 ? 2 : 3;",
     "case 4: return maxdeg == 3 ? 3 : 2;"),
    ("per-vertex triangles not halved", "tv[u - lo] = s / 2;", "tv[u - lo] = s;"),
    ("4-cycle rank test flipped", "if (dv > du || (dv == du && v > u)) continue;",
     "if (dv < du || (dv == du && v < u)) continue;"),
    ("clique order includes earlier neighbours", "if (key[u] > key[v]) L->col[w++] = u;",
     "if (key[u] != key[v]) L->col[w++] = u;"),
    ("ESU root test dropped", "if (u <= c->root) continue;", "if (u < 0) continue;"),
    ("ESU exclusive-neighbour test dropped", "if (near) continue;", "(void)near;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_reject_planted_mistake(tmp_path, name, old, new):
    """A plausible mistake planted in a copy of oracle.c must fail the pins."""
    import subprocess

    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", str(so), str(mut)])
    assert _pin_suite_passes(), "unmutated oracle must pass the compact pin suite"
    with oracle.use_variant(str(so)):
        assert not _pin_suite_passes(), f"pins did not catch: {name}"


# ------------------------------------------------------------ 5-vertex motifs
def test_p5_classes_known_census():
    """There are 21 connected graphs on 5 vertices: 3 trees and 5, 5, 4, 2, 1, 1
    graphs with 5..10 edges (the census of connected graphs)."""
    from collections import Counter

    codes = oracle.p5_classes()
    assert len(codes) == 21 and len(set(codes)) == 21
    assert sorted(Counter(bin(c).count("1") for c in codes).items()) == [
        (4, 3), (5, 5), (6, 5), (7, 4), (8, 2), (9, 1), (10, 1)]


def _p5_index(g5):
    """Output index of a connected 5-vertex graph (its one count)."""
    c = oracle.bf_motifs(g5, 5)
    assert sum(c) == 1
    return c.index(1)


def test_p5_closed_forms():
    import math

    star_i = _p5_index(gg.star(4))
    path_i = _p5_index(gg.path(5))
    k5_i = _p5_index(gg.complete(5))
    c5_i = _p5_index(gg.cycle(5))
    k23_i = _p5_index(gg.complete_multipartite((2, 3)))
    assert (path_i, star_i, c5_i, k5_i) == (0, 2, 3, 20)  # the order of the header comment
    for n in (5, 6, 9, 12):
        want = [0] * 21
        want[k5_i] = math.comb(n, 5)
        assert oracle.bf_motifs(gg.complete(n), 5) == want
    for s in (4, 7, 11):
        want = [0] * 21
        want[star_i] = math.comb(s, 4)
        assert oracle.bf_motifs(gg.star(s), 5) == want
    for n in (6, 9, 20):
        want = [0] * 21
        want[path_i] = n
        assert oracle.bf_motifs(gg.cycle(n), 5) == want
    for n in (5, 8, 30):
        want = [0] * 21
        want[path_i] = n - 4
        assert oracle.bf_motifs(gg.path(n), 5) == want
    for a, b in ((2, 3), (3, 4), (4, 6), (5, 5)):
        want = [0] * 21
        want[star_i] = a * math.comb(b, 4) + b * math.comb(a, 4)
        want[k23_i] = math.comb(a, 2) * math.comb(b, 3) + math.comb(a, 3) * math.comb(b, 2)
        assert oracle.bf_motifs(gg.complete_multipartite((a, b)), 5) == want


def test_p5_esu_agrees_with_brute_force():
    for i in range(40):
        g = gg.erdos_renyi(14 + i % 20, 0.12 + 0.02 * (i % 15), seed=900 + i)
        assert oracle.esu_motifs(g, 5) == oracle.bf_motifs(g, 5), g.name
    for g in (gg.barabasi_albert(60, 3, seed=3), gg.rmat(64, 300, seed=4)):
        assert oracle.esu_motifs(g, 5) == oracle.bf_motifs(g, 5)


def test_p5_relabel_invariance_and_roots():
    g = gg.barabasi_albert(300, 4, seed=8)
    perm = np.random.default_rng(1).permutation(g.n)
    assert oracle.esu_motifs(gg.relabel(g, perm), 5) == oracle.esu_motifs(g, 5)
    parts = [oracle.esu_motifs(g, 5, roots=r) for r in ((0, 100), (100, 101), (101, 300))]
    assert [sum(x) for x in zip(*parts)] == oracle.esu_motifs(g, 5)


def test_large_k_cliques():
    """k = 8..10 (the deepest levels the library counts): closed forms for
    complete and complete multipartite graphs, brute force (k = 8) and
    ID-order / degree-order agreement on dense small random graphs, and the join of an independent set A with a graph H,
    whose k-cliques are |A| * c_{k-1}(H) + c_k(H)."""
    for n in (10, 12, 14):
        g = gg.complete(n)
        for k in (8, 9, 10):
            assert oracle.clique_count(g, k, "id") == C(n, k)
            assert oracle.clique_count(g, k, "degree") == C(n, k)
    sizes = (2, 3, 2, 3, 2, 3, 2, 3, 2, 3, 1)
    g = gg.complete_multipartite(sizes)
    for k in (8, 9, 10):
        assert oracle.clique_count(g, k, "degree") == e_sym(sizes, k), k
    for seed in range(20):  # brute force goes to k = 8; ID and degree order agree beyond
        g = gg.erdos_renyi(14, 0.85, seed=500 + seed)
        assert oracle.clique_count(g, 8, "id") == oracle.bf_cliques(g, 8), seed
        for k in (8, 9, 10):
            assert oracle.clique_count(g, k, "id") == oracle.clique_count(g, k, "degree"), (seed, k)
    rng = np.random.default_rng(7)
    nb = 30
    iu = np.triu_indices(nb, 1)
    keep = rng.random(len(iu[0])) < 0.6
    h_edges = np.stack([iu[0][keep], iu[1][keep]], 1)
    h = gg.from_edges(nb, h_edges)
    join = np.stack(np.meshgrid(np.arange(nb), np.arange(nb, 2 * nb), indexing="ij"), -1).reshape(-1, 2)
    g = gg.from_edges(2 * nb, np.concatenate([join, h_edges + nb]))
    for k in (6, 8, 10):
        want = nb * oracle.clique_count(h, k - 1, "id") + oracle.clique_count(h, k, "id")
        assert oracle.clique_count(g, k, "degree") == want, k
