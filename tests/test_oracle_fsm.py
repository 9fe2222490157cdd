"""Pins of the oracle's frequent subgraph mining (oracle.fsm): edge-induced
embeddings of a vertex-labelled graph, MNI (domain) support (Sec. 2.1 FSM;
Sec. 3.3 Listing 5).

- Closed forms: K_n, stars, cycles, complete bipartite graphs with one label
  per side (counts and supports follow from the symmetry of these graphs).
- The textbook definition: MNI support by brute-force subgraph matching
  (oracle.fsm_bf_support, every injective label- and edge-preserving map)
  equals the oracle's support for every pattern it reports, on hundreds of
  small random labelled graphs; the matchings are a whole multiple of the
  embeddings (the automorphisms); and every labelled pattern of up to 3
  edges with a non-zero brute-force support is reported (completeness).
- Invariants: min_support keeps exactly the patterns at or above it; the
  support of a 2-edge pattern is at most that of each of its edges
  (anti-monotonicity); relabelling the vertices changes nothing.
- Planted mistakes in a copy of oracle.c are rejected by these pins.
"""
import itertools
import os
from math import comb as C

import numpy as np
import pytest

import graphgen as gg
import oracle

PAIRS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]  # adjacency bit i = pair i


def bits(edges):
    return sum(1 << PAIRS.index((min(a, b), max(a, b))) for a, b in edges)


def zeros(g):
    return np.zeros(g.n, np.int32)


def by_shape(res):
    """{(edges, nv): [(labels, support, embeddings)]} of an oracle result."""
    out = {}
    for p in res:
        out.setdefault((p["edges"], len(p["labels"])), []).append((p["labels"], p["support"], p["embeddings"]))
    return out


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_complete_graph(n):
    """K_n, one label: every vertex plays every role of every pattern."""
    s = by_shape(oracle.fsm(gg.complete(n), zeros(gg.complete(n)), 3))
    assert s[(1, 2)] == [((0, 0), n, C(n, 2))]
    assert s[(2, 3)] == [((0, 0, 0), n, n * C(n - 1, 2))]
    assert s[(3, 3)] == [((0, 0, 0), n, C(n, 3))]
    four = {lab_sup_cnt[2]: lab_sup_cnt for lab_sup_cnt in s[(3, 4)]}
    assert sorted(four) == sorted([n * C(n - 1, 3), n * (n - 1) * (n - 2) * (n - 3) // 2])  # stars, paths
    assert all(x[1] == n for x in s[(3, 4)])


@pytest.mark.parametrize("sz", [3, 4, 9])
def test_star(sz):
    """K_{1,s}: the centre is the only wedge/star centre (support 1); both
    ends of an edge share an orbit (support s + 1)."""
    g = gg.star(sz)
    s = by_shape(oracle.fsm(g, zeros(g), 3))
    assert s[(1, 2)] == [((0, 0), sz + 1, sz)]
    assert s[(2, 3)] == [((0, 0, 0), 1, C(sz, 2))]
    assert s[(3, 4)] == [((0, 0, 0, 0), 1, C(sz, 3))]
    assert (3, 3) not in s


@pytest.mark.parametrize("n", [5, 6, 11])
def test_cycle(n):
    g = gg.cycle(n)
    s = by_shape(oracle.fsm(g, zeros(g), 3))
    assert s[(1, 2)] == [((0, 0), n, n)]
    assert s[(2, 3)] == [((0, 0, 0), n, n)]
    assert s[(3, 4)] == [((0, 0, 0, 0), n, n)]  # 3-paths only
    assert (3, 3) not in s


@pytest.mark.parametrize("a,b", [(2, 3), (3, 3), (4, 6)])
def test_complete_bipartite_labelled(a, b):
    """K_{a,b}, label 0 on side A and 1 on side B."""
    g = gg.complete_multipartite((a, b))
    lab = np.array([0] * a + [1] * b, np.int32)
    res = oracle.fsm(g, lab, 3)
    got = {(p["labels"], p["adj"]): (p["support"], p["embeddings"]) for p in res}
    wedge, star, path = SHAPES["wedge"][1], SHAPES["star"][1], SHAPES["path"][1]
    want = {canon((0, 1), [(0, 1)]): (min(a, b), a * b),
            canon((0, 1, 1), wedge): (min(a, b), a * C(b, 2)),   # centre in A
            canon((1, 0, 0), wedge): (min(a, b), b * C(a, 2)),   # centre in B
            canon((0, 1, 0, 1), path): (min(a, b), a * b * (a - 1) * (b - 1))}
    if b >= 3:
        want[canon((0, 1, 1, 1), star)] = (min(a, b), a * C(b, 3))
    if a >= 3:
        want[canon((1, 0, 0, 0), star)] = (min(a, b), b * C(a, 3))
    assert got == want
    assert not any(p["edges"] == 3 and len(p["labels"]) == 3 for p in res)  # no triangles


# --------------------------------------------------- textbook definition
def canon(labels, edges):
    """Canonical (labels, bits) of a small labelled pattern by brute force."""
    nv = len(labels)
    best = None
    for p in itertools.permutations(range(nv)):
        pos = {v: i for i, v in enumerate(p)}
        cand = (tuple(labels[v] for v in p), bits([(pos[x], pos[y]) for x, y in edges]))
        best = cand if best is None or cand < best else best
    return best


SHAPES = {"edge": (2, [(0, 1)]), "wedge": (3, [(0, 1), (0, 2)]), "triangle": (3, [(0, 1), (0, 2), (1, 2)]),
          "star": (4, [(0, 1), (0, 2), (0, 3)]), "path": (4, [(0, 1), (1, 2), (2, 3)])}


def all_patterns(nlab):
    out = set()
    for nv, e in SHAPES.values():
        for labs in itertools.product(range(nlab), repeat=nv):
            out.add(canon(labs, e))
    return out


def random_labelled(count, nmax=9, nlab=3, seed=0):
    rng = np.random.default_rng(seed)
    for i in range(count):
        n = int(rng.integers(1, nmax + 1))
        p = float(rng.uniform(0.15, 0.8))
        g = gg.erdos_renyi(n, p, seed=1000 + i)
        yield g, rng.integers(0, nlab, size=n).astype(np.int32)


def test_brute_force_matching_agrees():
    cands = all_patterns(3)
    for g, lab in random_labelled(150):
        res = oracle.fsm(g, lab, 3)
        found = {}
        for p in res:
            sup, m = oracle.fsm_bf_support(g, lab, p["labels"], p["adj"])
            assert sup == p["support"], (g.name, p)
            assert p["embeddings"] >= 1 and m % p["embeddings"] == 0, (g.name, p, m)
            found[(p["labels"], p["adj"])] = p
        for labs, adj in cands:  # completeness: every occurring pattern is reported
            sup, m = oracle.fsm_bf_support(g, lab, labs, adj)
            assert (m > 0) == ((labs, adj) in found), (g.name, labs, adj)


def test_min_support_and_anti_monotonicity():
    for g, lab in random_labelled(40, nmax=14, nlab=2, seed=3):
        full = oracle.fsm(g, lab, 3)
        for sigma in (1, 2, 3, 5):
            assert oracle.fsm(g, lab, 3, sigma) == [p for p in full if p["support"] >= sigma]
        edge_sup = {p["labels"]: p["support"] for p in full if p["edges"] == 1}
        for p in full:
            if p["edges"] == 2:  # wedge: its centre is the vertex of degree 2
                labs, adj = p["labels"], p["adj"]
                deg = [sum(1 for i, (x, y) in enumerate(PAIRS) if adj >> i & 1 and v in (x, y)) for v in range(3)]
                c = deg.index(2)
                for e in (v for v in range(3) if v != c):
                    sub = tuple(sorted((labs[c], labs[e])))
                    assert edge_sup[sub] >= p["support"]
        assert oracle.fsm(g, lab, 2) == [p for p in full if p["edges"] <= 2]


def test_relabel_invariance():
    rng = np.random.default_rng(11)
    for g, lab in random_labelled(20, nmax=40, nlab=3, seed=5):
        perm = rng.permutation(g.n)
        h = gg.relabel(g, perm)
        lab2 = np.empty_like(lab)
        lab2[perm] = lab
        assert oracle.fsm(h, lab2, 3) == oracle.fsm(g, lab, 3)


# ------------------------------------------------ planted-mistake checks
def _fsm_pins_pass() -> bool:
    try:
        for n in (4, 6):
            g = gg.complete(n)
            s = by_shape(oracle.fsm(g, zeros(g), 3))
            if s.get((3, 3)) != [((0, 0, 0), n, C(n, 3))] or s.get((2, 3)) != [((0, 0, 0), n, n * C(n - 1, 2))]:
                return False
            if sorted(x[2] for x in s.get((3, 4), [])) != sorted([n * C(n - 1, 3), n * (n - 1) * (n - 2) * (n - 3) // 2]):
                return False
        g = gg.star(5)
        s = by_shape(oracle.fsm(g, zeros(g), 3))
        if s.get((1, 2)) != [((0, 0), 6, 5)] or (3, 3) in s:
            return False
        for g, lab in random_labelled(40, seed=9):
            for p in oracle.fsm(g, lab, 3):
                if oracle.fsm_bf_support(g, lab, p["labels"], p["adj"])[0] != p["support"]:
                    return False
    except RuntimeError:
        return False
    return True


MUTATIONS = [
    ("orbit union dropped", "if (p[i] < orb[i]) orb[i] = p[i];", "(void)p;"),
    ("path counted from both middle arcs", "if (max_edges < 3 || c < u) continue;", "if (max_edges < 3) continue;"),
    ("triangle closure test dropped", "if (N[i] > u && adjacent(rp, col, N[i], N[j])) {", "if (N[i] > u) {"),
    ("path end may repeat", "if (b == u || b == a) continue;", "if (b == u) continue;"),
    ("support as the largest domain", "if (d < sup) sup = d;", "if (sup == UINT64_MAX || d > sup) sup = d;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_fsm_pins_reject_planted_mistake(tmp_path, name, old, new):
    import subprocess

    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", str(so), str(mut)])
    assert _fsm_pins_pass(), "unmutated oracle must pass the compact pin suite"
    with oracle.use_variant(str(so)):
        assert not _fsm_pins_pass(), f"pins did not catch: {name}"
