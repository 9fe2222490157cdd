"""CPU oracle for k-clique and k-motif counts -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  It is independent of the CUDA
library: it shares no code, header, table or constant with it and does not
import it.  The C source (``oracle.c``) is compiled with gcc into
``liboracle.so`` next to this file.

Functions and the passages they follow:

* ``bf_cliques`` / ``bf_motifs`` -- brute force over every k-subset (n <= 64):
  the definitions of Sec. 2.1-2.2 (clique = pairwise adjacent vertex set;
  motif = isomorphism class of a connected vertex-induced subgraph).
* ``clique_count`` -- plain depth-first clique enumerator (vertex-ID order or
  (degree, ID) order), per-size counts of every clique level.
* ``esu_motifs`` -- ESU enumeration (Wernicke 2006) of connected k-sets.
* ``formula_motifs`` -- special-pattern counts plus pattern relationships
  (the "eliding isomorphism test" idea of Sec. 2.2).
* ``fsm`` -- frequent subgraph mining (Sec. 2.1 FSM, Sec. 3.3 Listing 5):
  connected edge sets of 1..3 edges enumerated once by shape, canonical
  labelled patterns by brute force over vertex orders, MNI support from the
  (pattern, automorphism orbit, vertex) triples; ``fsm_bf_support`` -- MNI
  by brute-force subgraph matching (its textbook definition).
* ``exclusive_scan`` -- the prefix-sum step of inspection-execution
  (Sec. 5.3); ``connectivity_mask`` -- the binary-search connectivity check
  (Sec. 5.4).

Pins (see ``tests/test_oracle.py``): closed forms on complete, complete
multipartite, star, cycle, path and complete bipartite graphs; the degree
identities; brute force on small random graphs; relabelling invariance;
agreement between tiers; the paper's worked examples (Sec. 5.3, Sec. 5.4).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MOTIF3 = ("wedge", "triangle")
MOTIF4 = ("3-star", "4-path", "tailed-triangle", "4-cycle", "diamond", "4-clique")

_ERR = {-1: "invalid argument", -3: "out of memory", -6: "count overflows uint64"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (in-tree) when missing or stale."""
    with open(_SRC, "rb") as f:
        dig = hashlib.sha256(f.read()).hexdigest()[:16]
    stamp = _LIB + ".src"
    if not force and os.path.exists(_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return _LIB


_lib = None


def _declare(lib):
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.orc_bf_cliques.restype = I32
    lib.orc_bf_cliques.argtypes = [I32, P, P, I32, P]
    lib.orc_bf_motifs.restype = I32
    lib.orc_bf_motifs.argtypes = [I32, P, P, I32, P]
    lib.orc_clique_count.restype = I32
    lib.orc_clique_count.argtypes = [I32, P, P, I32, I32, I32, I32, I32, P]
    lib.orc_p5_classes.restype = I32
    lib.orc_p5_classes.argtypes = [P]
    lib.orc_esu_motifs.restype = I32
    lib.orc_esu_motifs.argtypes = [I32, P, P, I32, I32, I32, I32, P]
    lib.orc_formula_motifs_range.restype = I32
    lib.orc_formula_motifs_range.argtypes = [I32, P, P, I32, I32, I32, I32, P]
    lib.orc_formula_motifs_batch.restype = I32
    lib.orc_formula_motifs_batch.argtypes = [I32, P, P, I32, P, I32, P]
    lib.orc_exclusive_scan.argtypes = [I64, P, P]
    lib.orc_connectivity_mask.restype = ctypes.c_uint32
    lib.orc_connectivity_mask.argtypes = [P, P, I32, P, I32]
    lib.orc_degree_sums.argtypes = [I32, P, P, P, P]
    lib.orc_fsm.restype = I32
    lib.orc_fsm.argtypes = [I32, P, P, P, I32, I64, P, P, I32, P]
    lib.orc_fsm_bf_support.restype = I32
    lib.orc_fsm_bf_support.argtypes = [I32, P, P, P, I32, P, I32, P, P]
    return lib


_override = None


def _L():
    """The loaded oracle library (or a variant installed by ``use_variant``)."""
    global _lib
    if _override is not None:
        return _override
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


class use_variant:
    """Context manager: route every oracle call to another build of oracle.c.

    Used only by the planted-mistake tests, which compile a mutated copy of
    the source and check that the pins reject it.
    """

    def __init__(self, so_path: str):
        self.lib = _declare(ctypes.CDLL(so_path))

    def __enter__(self):
        global _override
        _override = self.lib
        return self

    def __exit__(self, *exc):
        global _override
        _override = None
        return False


def _arrs(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return rp, col


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what}: {_ERR.get(rc, rc)}")


def bf_cliques(g, k: int) -> int:
    rp, col = _arrs(g)
    out = np.zeros(1, np.uint64)
    _check(_L().orc_bf_cliques(g.n, rp.ctypes.data, col.ctypes.data, k, out.ctypes.data), "bf_cliques")
    return int(out[0])


def _npat(k: int) -> int:
    return {3: 2, 4: 6, 5: 21}[k]


def bf_motifs(g, k: int) -> list:
    rp, col = _arrs(g)
    out = np.zeros(21, np.uint64)
    _check(_L().orc_bf_motifs(g.n, rp.ctypes.data, col.ctypes.data, k, out.ctypes.data), "bf_motifs")
    return [int(x) for x in out[: _npat(k)]]


def p5_classes() -> list:
    """Canonical 10-bit adjacency codes of the connected 5-vertex classes, in output order."""
    codes = np.zeros(64, np.int32)
    n = _L().orc_p5_classes(codes.ctypes.data)
    return [int(x) for x in codes[:n]]


def clique_levels(g, k: int, order: str = "id", roots=None, threads: int = 1) -> list:
    """Counts of l-cliques for l = 1..k (index l) with first vertex in ``roots``."""
    rp, col = _arrs(g)
    lo, hi = (0, g.n) if roots is None else roots
    out = np.zeros(k + 1, np.uint64)
    rc = _L().orc_clique_count(g.n, rp.ctypes.data, col.ctypes.data, k, 1 if order == "degree" else 0,
                               lo, hi, threads, out.ctypes.data)
    _check(rc, "clique_count")
    return [int(x) for x in out]


def clique_count(g, k: int, order: str = "id", threads: int = 1) -> int:
    return clique_levels(g, k, order, None, threads)[k]


def esu_motifs(g, k: int, roots=None, threads: int = 1) -> list:
    rp, col = _arrs(g)
    lo, hi = (0, g.n) if roots is None else roots
    out = np.zeros(21, np.uint64)
    rc = _L().orc_esu_motifs(g.n, rp.ctypes.data, col.ctypes.data, k, lo, hi, threads, out.ctypes.data)
    _check(rc, "esu_motifs")
    return [int(x) for x in out[: _npat(k)]]


def formula_motifs(g, k: int, threads: int = 1) -> list:
    rp, col = _arrs(g)
    out = np.zeros(6, np.uint64)
    rc = _L().orc_formula_motifs_range(g.n, rp.ctypes.data, col.ctypes.data, 0, g.n, k, threads,
                                       out.ctypes.data)
    _check(rc, "formula_motifs")
    return [int(x) for x in out[: (2 if k == 3 else 6)]]


def formula_motifs_batch(batch, k: int) -> np.ndarray:
    """Per-graph motif counts of a disjoint-union batch, shape (G, 2 or 6)."""
    rp, col = _arrs(batch.graph)
    vo = np.ascontiguousarray(batch.vtx_off, dtype=np.int64)
    np_ = 2 if k == 3 else 6
    out = np.zeros((batch.G, np_), np.uint64)
    rc = _L().orc_formula_motifs_batch(batch.graph.n, rp.ctypes.data, col.ctypes.data, batch.G,
                                       vo.ctypes.data, k, out.ctypes.data)
    _check(rc, "formula_motifs_batch")
    return out


def fsm(g, labels, max_edges: int, min_support: int = 0) -> list:
    """Frequent edge-induced labelled patterns of 1..max_edges (<= 3) edges
    with MNI support >= min_support (Sec. 2.1, Sec. 3.3 Listing 5), ordered
    by (edges, vertices, labels, adjacency); each a dict with the canonical
    pattern (vertex labels and adjacency bits over the pairs (0,1), (0,2),
    (0,3), (1,2), (1,3), (2,3) in the order that makes (labels, bits)
    smallest), its support and its number of embeddings."""
    rp, col = _arrs(g)
    lab = np.ascontiguousarray(labels, np.int32)
    assert lab.shape[0] == g.n
    n = ctypes.c_int32()
    _check(_L().orc_fsm(g.n, rp.ctypes.data, col.ctypes.data, lab.ctypes.data, max_edges, min_support,
                        None, None, 0, ctypes.byref(n)), "fsm")
    cap = max(n.value, 1)
    meta = np.zeros((cap, 7), np.int32)
    val = np.zeros((cap, 2), np.uint64)
    _check(_L().orc_fsm(g.n, rp.ctypes.data, col.ctypes.data, lab.ctypes.data, max_edges, min_support,
                        meta.ctypes.data, val.ctypes.data, cap, ctypes.byref(n)), "fsm")
    out = []
    for r in range(n.value):
        nv = int(meta[r, 1])
        out.append({"edges": int(meta[r, 0]), "labels": tuple(int(x) for x in meta[r, 2:2 + nv]),
                    "adj": int(meta[r, 6]), "support": int(val[r, 0]), "embeddings": int(val[r, 1])})
    return out


def fsm_bf_support(g, labels, plabels, padj: int):
    """(MNI support, matchings) of one pattern by brute-force subgraph
    matching, the textbook definition (n <= 64)."""
    rp, col = _arrs(g)
    lab = np.ascontiguousarray(labels, np.int32)
    pl = np.ascontiguousarray(plabels, np.int32)
    s, m = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_L().orc_fsm_bf_support(g.n, rp.ctypes.data, col.ctypes.data, lab.ctypes.data, len(pl), pl.ctypes.data,
                                   padj, ctypes.byref(s), ctypes.byref(m)), "fsm_bf_support")
    return int(s.value), int(m.value)


def exclusive_scan(counts) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.zeros(c.size + 1, np.int64)
    _L().orc_exclusive_scan(c.size, c.ctypes.data, out.ctypes.data)
    return out


def connectivity_mask(g, emb, u: int) -> int:
    rp, col = _arrs(g)
    e = np.ascontiguousarray(emb, dtype=np.int32)
    return int(_L().orc_connectivity_mask(rp.ctypes.data, col.ctypes.data, e.size, e.ctypes.data, u))


def degree_sums(g):
    """(sum_v C(d_v, 2), sum_v C(d_v, 3), max degree) as Python ints."""
    rp, _ = _arrs(g)
    c2 = np.zeros(2, np.uint64)
    c3 = np.zeros(2, np.uint64)
    dm = np.zeros(1, np.int64)
    _L().orc_degree_sums(g.n, rp.ctypes.data, c2.ctypes.data, c3.ctypes.data, dm.ctypes.data)
    return int(c2[0]) | (int(c2[1]) << 64), int(c3[0]) | (int(c3[1]) << 64), int(dm[0])
