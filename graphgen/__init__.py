"""Seeded synthetic graphs in CSR form (inputs only).

This module produces the inputs that both the CPU oracle and the CUDA path
consume.  It contains no pattern-mining arithmetic: only random-graph
generators (``gen.c``), a CSR container and a small on-disk cache.

Every graph is undirected and simple (symmetric, sorted neighbour lists, no
self-loops, no duplicate edges), the input format the paper assumes (Sec. 6.1,
experimental setup).  Vertex IDs are int32, row pointers int64.

The named workloads mirror the shapes of the paper's inputs (Sec. 6.1,
Table 1: power-law graphs with millions of vertices and average degree around
10-27), since the paper's datasets themselves are not available here.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_CACHE = os.environ.get("PGM_GRAPH_CACHE", os.path.join(os.path.dirname(_HERE), ".graphcache"))

RMAT_ABC = (0.57, 0.19, 0.19)


@dataclass
class CSR:
    """Undirected simple graph: ``rowptr`` (int64, n+1) and ``col`` (int32)."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    name: str = ""

    @property
    def narcs(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        return self.narcs // 2


@dataclass
class Batch:
    """Disjoint union of G graphs; graph i owns vertices [vtx_off[i], vtx_off[i+1])."""

    vtx_off: np.ndarray
    graph: CSR
    kind: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    param: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))

    @property
    def G(self) -> int:
        return int(self.vtx_off.shape[0] - 1)

    def part(self, i: int) -> CSR:
        """Graph i alone, relabelled to local vertex IDs."""
        v0, v1 = int(self.vtx_off[i]), int(self.vtx_off[i + 1])
        rp = self.graph.rowptr[v0 : v1 + 1]
        col = self.graph.col[rp[0] : rp[-1]] - v0
        return CSR(v1 - v0, (rp - rp[0]).astype(np.int64), col.astype(np.int32), f"part{i}")


# ------------------------------------------------------------------ build
def _src_digest() -> str:
    with open(_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def build(force: bool = False) -> str:
    """Compile gen.c into libgraphgen.so (in-tree) when missing or stale."""
    stamp = _LIB + ".src"
    dig = _src_digest()
    if not force and os.path.exists(_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, U64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gg_graph_n.restype = I64
        lib.gg_graph_n.argtypes = [P]
        lib.gg_graph_narcs.restype = I64
        lib.gg_graph_narcs.argtypes = [P]
        lib.gg_graph_copy.argtypes = [P, P, P]
        lib.gg_graph_free.argtypes = [P]
        lib.gg_from_edges.restype = P
        lib.gg_from_edges.argtypes = [I64, I64, P, P]
        lib.gg_er.restype = P
        lib.gg_er.argtypes = [I64, D, U64, U64]
        lib.gg_rmat.restype = P
        lib.gg_rmat.argtypes = [I64, I64, D, D, D, U64, U64]
        lib.gg_chung_lu.restype = P
        lib.gg_chung_lu.argtypes = [I64, D, D, D, U64, U64]
        lib.gg_ba.restype = P
        lib.gg_ba.argtypes = [I64, I64, U64, U64]
        lib.gg_batch_small.restype = P
        lib.gg_batch_small.argtypes = [I64, I64, I64, D, D, I64, I64, U64]
        lib.gg_batch_mixed.restype = P
        lib.gg_batch_mixed.argtypes = [I64, I64, I64, D, D, D, D, D, U64]
        lib.gg_batch_G.restype = I64
        lib.gg_batch_G.argtypes = [P]
        lib.gg_batch_graph.restype = P
        lib.gg_batch_graph.argtypes = [P]
        lib.gg_batch_copy_meta.argtypes = [P, P, P, P]
        lib.gg_batch_free.argtypes = [P]
        lib.gg_poisson_stream.argtypes = [I64, D, I64, I64, U64, P, P, P]
        _lib = lib
    return _lib


def _take_graph(h, name: str, free: bool = True) -> CSR:
    if not h:
        raise RuntimeError(f"graph generation failed: {name}")
    lib = _L()
    n = lib.gg_graph_n(h)
    na = lib.gg_graph_narcs(h)
    rowptr = np.empty(n + 1, np.int64)
    col = np.empty(max(na, 1), np.int32)
    lib.gg_graph_copy(h, rowptr.ctypes.data, col.ctypes.data)
    if free:
        lib.gg_graph_free(h)
    return CSR(int(n), rowptr, col[:na], name)


# ------------------------------------------------------------- generators
def from_edges(n: int, edges, name: str = "edges") -> CSR:
    """Simple symmetric CSR from an undirected edge list (loops/dups dropped)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    us = np.ascontiguousarray(e[:, 0])
    vs = np.ascontiguousarray(e[:, 1])
    return _take_graph(_L().gg_from_edges(n, e.shape[0], us.ctypes.data, vs.ctypes.data), name)


def erdos_renyi(n: int, p: float, seed: int = 1, stream: int = 0) -> CSR:
    return _take_graph(_L().gg_er(n, p, seed, stream), f"er_n{n}_p{p:.6g}_s{seed}")


def rmat(n: int, m: int, abc=RMAT_ABC, seed: int = 1, stream: int = 0) -> CSR:
    a, b, c = abc
    return _take_graph(_L().gg_rmat(n, m, a, b, c, seed, stream), f"rmat_n{n}_m{m}_s{seed}")


def chung_lu(n: int, gamma: float, mean_deg: float, wmax: float, seed: int = 1, stream: int = 0) -> CSR:
    return _take_graph(
        _L().gg_chung_lu(n, gamma, mean_deg, wmax, seed, stream), f"cl_n{n}_g{gamma}_d{mean_deg}_s{seed}"
    )


def barabasi_albert(n: int, m: int, seed: int = 1, stream: int = 0) -> CSR:
    return _take_graph(_L().gg_ba(n, m, seed, stream), f"ba_n{n}_m{m}_s{seed}")


def _take_batch(h, name: str) -> Batch:
    if not h:
        raise RuntimeError(f"batch generation failed: {name}")
    lib = _L()
    G = lib.gg_batch_G(h)
    vo = np.empty(G + 1, np.int64)
    kind = np.empty(max(G, 1), np.int32)
    param = np.empty(max(G, 1), np.float64)
    lib.gg_batch_copy_meta(h, vo.ctypes.data, kind.ctypes.data, param.ctypes.data)
    g = _take_graph(lib.gg_batch_graph(h), name, free=False)
    lib.gg_batch_free(h)
    return Batch(vo, g, kind[:G], param[:G])


def batch_small(G: int, nmin=16, nmax=4096, dmin=4.0, dmax=32.0, mmin=2, mmax=8, seed: int = 1) -> Batch:
    """G small graphs: even i Erdos-Renyi, odd i Barabasi-Albert."""
    return _take_batch(
        _L().gg_batch_small(G, nmin, nmax, dmin, dmax, mmin, mmax, seed), f"batch_small_G{G}_s{seed}"
    )


def batch_mixed(G: int, nmin=1000, nmax=1_000_000, dmin=8.0, dmax=32.0, abc=RMAT_ABC, seed: int = 1) -> Batch:
    """G resident graphs: first half R-MAT, second half Barabasi-Albert."""
    a, b, c = abc
    return _take_batch(
        _L().gg_batch_mixed(G, nmin, nmax, dmin, dmax, a, b, c, seed), f"batch_mixed_G{G}_s{seed}"
    )


def poisson_stream(count: int, lam: float, ntypes: int, ngraphs: int, seed: int = 1):
    """Arrival times (s), query types and target graphs of a Poisson request stream."""
    t = np.empty(count, np.float64)
    q = np.empty(count, np.int32)
    g = np.empty(count, np.int32)
    _L().gg_poisson_stream(count, lam, ntypes, ngraphs, seed, t.ctypes.data, q.ctypes.data, g.ctypes.data)
    return t, q, g


# --------------------------------------------------------- special graphs
def complete(n: int) -> CSR:
    iu = np.triu_indices(n, 1)
    return from_edges(n, np.stack(iu, 1), f"K{n}")


def complete_multipartite(sizes) -> CSR:
    part = np.repeat(np.arange(len(sizes)), sizes)
    n = int(part.shape[0])
    iu = np.triu_indices(n, 1)
    keep = part[iu[0]] != part[iu[1]]
    return from_edges(n, np.stack([iu[0][keep], iu[1][keep]], 1), f"K{'_'.join(map(str, sizes))}")


def star(s: int) -> CSR:
    return from_edges(s + 1, [(0, i) for i in range(1, s + 1)], f"star{s}")


def cycle(n: int) -> CSR:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def path(n: int) -> CSR:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"P{n}")


def empty(n: int) -> CSR:
    return CSR(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), f"empty{n}")


def relabel(g: CSR, perm) -> CSR:
    """The same graph with vertex v renamed perm[v]."""
    perm = np.asarray(perm, np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    e = np.stack([perm[src], perm[g.col.astype(np.int64)]], 1)
    e = e[e[:, 0] < e[:, 1]]
    return from_edges(g.n, e, g.name + "_relab")


def disjoint_union(graphs) -> Batch:
    """Concatenate graphs into one batch (global vertex IDs)."""
    vo = [0]
    rps, cols = [], []
    a = 0
    for g in graphs:
        rps.append(g.rowptr[:-1] + a)
        cols.append(g.col.astype(np.int64) + vo[-1])
        a += g.narcs
        vo.append(vo[-1] + g.n)
    rowptr = np.concatenate(rps + [np.array([a], np.int64)]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return Batch(np.array(vo, np.int64), CSR(vo[-1], rowptr, col, "union"))


# ------------------------------------------------------- named workloads
def _cached(key: str, make):
    os.makedirs(_CACHE, exist_ok=True)
    tag = hashlib.sha256((key + _src_digest()).encode()).hexdigest()[:20]
    path_ = os.path.join(_CACHE, f"{key}_{tag}.npz")
    if os.path.exists(path_):
        z = np.load(path_)
        if "vtx_off" in z:
            return Batch(z["vtx_off"], CSR(int(z["n"]), z["rowptr"], z["col"], key), z["kind"], z["param"])
        return CSR(int(z["n"]), z["rowptr"], z["col"], key)
    obj = make()
    tmp = path_ + f".tmp{os.getpid()}.npz"
    if isinstance(obj, Batch):
        np.savez(tmp, n=obj.graph.n, rowptr=obj.graph.rowptr, col=obj.graph.col,
                 vtx_off=obj.vtx_off, kind=obj.kind, param=obj.param)
    else:
        np.savez(tmp, n=obj.n, rowptr=obj.rowptr, col=obj.col)
    os.replace(tmp, path_)
    if isinstance(obj, Batch):
        obj.graph.name = key
    else:
        obj.name = key
    return obj


def triangle_er(seed: int = 1) -> CSR:
    """Erdos-Renyi, n = 4096, p = 16/4095 (average degree 16)."""
    return _cached(f"er4096_s{seed}", lambda: erdos_renyi(4096, 16.0 / 4095.0, seed))


def rmat21(seed: int = 1) -> CSR:
    """R-MAT scale 21 (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), exactly 28,000,000 edges."""
    return _cached(f"rmat21_m28M_s{seed}", lambda: rmat(1 << 21, 28_000_000, RMAT_ABC, seed))


def chung_lu_1m(seed: int = 1) -> CSR:
    """Chung-Lu, n = 2^20, exponent 2.1, mean weight 10, weights capped at 20,000."""
    return _cached(f"cl1m_s{seed}", lambda: chung_lu(1 << 20, 2.1, 10.0, 20000.0, seed))


def small_batch_20k(seed: int = 1) -> Batch:
    """20,000 graphs, n uniform in [16, 4096]; half ER (degree 4-32), half BA (m 2-8)."""
    return _cached(f"batch20k_s{seed}", lambda: batch_small(20000, seed=seed))


def serving_64(seed: int = 1) -> Batch:
    """64 resident graphs (32 R-MAT, 32 BA), n log-uniform in [1e3, 1e6], degree 8-32."""
    return _cached(f"serve64_s{seed}", lambda: batch_mixed(64, seed=seed))


def rmat_weak(scale: int, seed: int = 1) -> CSR:
    """R-MAT of the weak-scaling series: 2^scale vertices, average degree 20
    (10 * 2^scale undirected edges), same (a, b, c, d) as the R-MAT workload."""
    return _cached(f"rmat{scale}_d20_s{seed}", lambda: rmat(1 << scale, 10 << scale, RMAT_ABC, seed))


# ------------------------------------------------------------ vertex labels
def vertex_labels(n: int, nlabels: int, seed: int = 1, skew: float = 0.0) -> np.ndarray:
    """Seeded vertex labels in [0, nlabels) (int32[n]): uniform, or with
    P(label i) proportional to (i + 1)^-skew -- the uneven label frequencies
    of the labelled graphs that frequent subgraph mining runs on."""
    rng = np.random.default_rng(seed)
    if skew <= 0.0:
        return rng.integers(0, nlabels, size=n).astype(np.int32)
    p = (np.arange(1, nlabels + 1, dtype=np.float64)) ** -skew
    return rng.choice(nlabels, size=n, p=p / p.sum()).astype(np.int32)


def mico_like(seed: int = 1) -> CSR:
    """Stand-in for the paper's Mico input (Table 1: 100,000 vertices,
    2,160,312 arcs, average degree 22, 29 labels): Chung-Lu, n = 100,000,
    exponent 2.1, mean weight 21.6, weights capped at 1,359; its labels are
    vertex_labels(n, 29, seed, skew=1.0)."""
    return _cached(f"micolike_s{seed}", lambda: chung_lu(100_000, 2.1, 21.6, 1359.0, seed))


def youtube_like(seed: int = 1) -> CSR:
    """Stand-in for the paper's Youtube input (Table 1: 7,066,392 vertices,
    114,190,484 arcs, average degree 16, 29 labels): Chung-Lu, n =
    7,066,392, exponent 2.2, mean weight 16.2, weights capped at 2,000; its
    labels are vertex_labels(n, 29, seed, skew=1.0)."""
    return _cached(f"youtubelike_s{seed}", lambda: chung_lu(7_066_392, 2.2, 16.2, 2000.0, seed))


def patent_like(seed: int = 1) -> CSR:
    """Stand-in for the paper's Patents input (Table 1: 2,745,761 vertices,
    27,930,818 arcs, average degree 10, 37 labels): Chung-Lu, n = 2,745,761,
    exponent 2.5, mean weight 10.2, weights capped at 800; its labels are
    vertex_labels(n, 37, seed, skew=1.0)."""
    return _cached(f"patentlike_s{seed}", lambda: chung_lu(2_745_761, 2.5, 10.2, 800.0, seed))
