"""ctypes binding of libpgm (include/pgm.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls, converts
numpy arrays / Python ints into the C arguments, raises ``PgmError`` when the
call does not return ``PGM_OK`` and returns the output arguments.  No step of
the computation happens in Python, and there is no fallback: if
``libpgm.so`` is missing or no CUDA device is usable the calls fail.

Streams may be given as a ``torch.cuda.Stream``, a raw ``cudaStream_t``
integer, or ``None`` (the legacy default stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PGM_LIB=debug loads the bounds-checked build (libpgm_debug.so, see build.py)
LIB_PATH = os.path.join(_HERE, "libpgm_debug.so" if os.environ.get("PGM_LIB") == "debug" else "libpgm.so")

PGM_OK = 0
PGM_EINVAL = -1
PGM_EUNSUPPORTED = -2
PGM_ENOMEM = -3
PGM_ECUDA = -4
PGM_ETIMEOUT = -5
PGM_EOVERFLOW = -6
PGM_EBUSY = -7
STATUS_NAMES = {0: "PGM_OK", -1: "PGM_EINVAL", -2: "PGM_EUNSUPPORTED", -3: "PGM_ENOMEM",
                -4: "PGM_ECUDA", -5: "PGM_ETIMEOUT", -6: "PGM_EOVERFLOW", -7: "PGM_EBUSY"}

PGM_VALIDATE = 1
PGM_SANITIZE = 2

PGM_Q_TRIANGLE = 0
PGM_Q_KCLIQUE = 1
PGM_Q_MOTIF = 2

MOTIF3 = ("wedge", "triangle")
MOTIF4 = ("3-star", "4-path", "tailed-triangle", "4-cycle", "diamond", "4-clique")


class PgmError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pgm_graph_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("dmax", C.c_int64), ("dag_dmax", C.c_int64),
                ("sum_c2", C.c_uint64 * 2), ("sum_c3", C.c_uint64 * 2)]


class pgm_options(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("warp_stage_cap", C.c_int32), ("hub_threshold", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("level_budget", C.c_int64), ("profile", C.c_int32),
                ("reverse_ratio", C.c_int32), ("clique_engine", C.c_int32),
                ("bitset_forward_ratio", C.c_int32), ("bitset_smem_degree", C.c_int32),
                ("motif_order", C.c_int32), ("count_headroom_log2", C.c_int32), ("motif_b_side_min", C.c_int32),
                ("fsm_domain_order", C.c_int32)]


class pgm_phase(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("level", C.c_int32), ("launches", C.c_int32), ("ms", C.c_double),
                ("entries", C.c_double), ("alg_bytes", C.c_double)]


class pgm_profile(C.Structure):
    _fields_ = [("nphases", C.c_int32), ("phase", pgm_phase * 64), ("level_size", C.c_uint64 * 16),
                ("chunks", C.c_int32)]


class pgm_tune(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("warp_stage_cap", C.c_int32), ("hub_threshold", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("use_graph", C.c_int32), ("motif_b_side_min", C.c_int32),
                ("reverse_ratio", C.c_int32), ("bitset_forward_ratio", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class pgm_tune_trial(C.Structure):
    _fields_ = [("tune", pgm_tune), ("ms", C.c_double)]


class pgm_query(C.Structure):
    _fields_ = [("kind", C.c_int32), ("k", C.c_int32), ("graph", C.c_int32), ("pad", C.c_int32)]


class pgm_result(C.Structure):
    _fields_ = [("done", C.c_int32), ("status", C.c_int32), ("counts", C.c_uint64 * 6), ("submit_s", C.c_double),
                ("start_s", C.c_double), ("finish_s", C.c_double), ("mem_bytes", C.c_int64)]


class pgm_fsm_pattern(C.Structure):
    _fields_ = [("edges", C.c_int32), ("nv", C.c_int32), ("labels", C.c_int32 * 4), ("adj", C.c_uint32),
                ("pad", C.c_uint32), ("support", C.c_uint64), ("embeddings", C.c_uint64)]


P = C.c_void_p
_SIGS = {
    "pgm_graph_create_csr": (C.c_int, [C.c_int32, P, P, C.c_uint32, P, C.POINTER(P)]),
    "pgm_graph_create_csr_dev": (C.c_int, [C.c_int32, P, P, C.c_int64, C.c_uint32, P, C.POINTER(P)]),
    "pgm_graph_orient_by_degree": (C.c_int, [P]),
    "pgm_graph_stats_get": (C.c_int, [P, C.POINTER(pgm_graph_stats)]),
    "pgm_graph_destroy": (None, [P]),
    "pgm_count_kcliques": (C.c_int, [P, C.c_int32, C.POINTER(C.c_uint64)]),
    "pgm_count_kcliques_range": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_uint64)]),
    "pgm_list_kcliques": (C.c_int, [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    "pgm_list_motifs": (C.c_int, [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    "pgm_list_kcliques_host": (C.c_int, [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    "pgm_list_motifs_host": (C.c_int, [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]),
    "pgm_count_motifs": (C.c_int, [P, C.c_int32, P, C.c_int32]),
    "pgm_count_motifs_range": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, P, C.c_int32]),
    "pgm_batch_create": (C.c_int, [C.c_int32, P, P, P, C.c_uint32, P, C.POINTER(P)]),
    "pgm_batch_count_motifs": (C.c_int, [P, C.c_int32, P, C.POINTER(pgm_tune)]),
    "pgm_batch_count_kcliques": (C.c_int, [P, C.c_int32, P, C.POINTER(pgm_tune)]),
    "pgm_batch_count_motifs_loop": (C.c_int, [P, C.c_int32, P]),
    "pgm_batch_autotune": (C.c_int, [P, C.c_int32, C.POINTER(pgm_tune), C.POINTER(C.c_double)]),
    "pgm_batch_autotune_ex": (C.c_int, [P, C.c_int32, C.c_char_p, C.POINTER(pgm_tune), C.POINTER(C.c_double),
                                        C.POINTER(pgm_tune_trial), C.c_int32, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32)]),
    "pgm_batch_size": (C.c_int32, [P]),
    "pgm_batch_destroy": (None, [P]),
    "pgm_server_create": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(P)]),
    "pgm_server_add_graph": (C.c_int, [P, C.c_int32, P, P, C.POINTER(C.c_int32)]),
    "pgm_server_submit": (C.c_int, [P, C.POINTER(pgm_query), C.POINTER(C.c_int64)]),
    "pgm_server_poll": (C.c_int, [P, C.c_int64, C.POINTER(pgm_result)]),
    "pgm_server_drain": (C.c_int, [P, C.c_double]),
    "pgm_server_destroy": (None, [P]),
    "pgm_set_options": (C.c_int, [C.POINTER(pgm_options)]),
    "pgm_get_options": (C.c_int, [C.POINTER(pgm_options)]),
    "pgm_last_profile": (C.c_int, [C.POINTER(pgm_profile)]),
    "pgm_exclusive_scan_dev": (C.c_int, [P, C.c_int64, P, P]),
    "pgm_last_error": (C.c_char_p, []),
    "pgm_version": (C.c_char_p, []),
    "pgm_kernel_launches": (C.c_uint64, []),
    "pgm_debug_errors": (C.c_uint64, [C.c_int32]),
    "pgm_count_triangles_noalloc": (C.c_int, [C.c_int32, P, P, C.c_int64, P, P]),
    "pgm_graph_set_labels": (C.c_int, [P, P]),
    "pgm_fsm": (C.c_int, [P, C.c_int32, C.c_int64, C.POINTER(pgm_fsm_pattern), C.c_int32, C.POINTER(C.c_int32)]),
}

_lib = None


def load() -> C.CDLL:
    """Load libpgm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1911_06969_b300.build`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _stream(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _ok(rc: int, func: str):
    if rc != PGM_OK:
        raise PgmError(rc, func, load().pgm_last_error().decode(errors="replace"))


def _host_csr(rowptr, col):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    if cl.size == 0:
        cl = np.zeros(1, np.int32)
    return rp, cl


# ------------------------------------------------------------------ graphs
def pgm_graph_create_csr(n: int, rowptr, col, flags: int = 0, stream=None) -> int:
    rp, cl = _host_csr(rowptr, col)
    h = P()
    _ok(load().pgm_graph_create_csr(n, rp.ctypes.data, cl.ctypes.data, flags, _stream(stream), C.byref(h)),
        "pgm_graph_create_csr")
    return h.value


def pgm_graph_create_csr_dev(n: int, rowptr_dev_ptr: int, col_dev_ptr: int, narcs: int, flags: int = 0,
                             stream=None) -> int:
    h = P()
    _ok(load().pgm_graph_create_csr_dev(n, rowptr_dev_ptr, col_dev_ptr, narcs, flags, _stream(stream),
                                        C.byref(h)), "pgm_graph_create_csr_dev")
    return h.value


def pgm_graph_orient_by_degree(g: int):
    _ok(load().pgm_graph_orient_by_degree(g), "pgm_graph_orient_by_degree")


def pgm_graph_stats_get(g: int) -> dict:
    s = pgm_graph_stats()
    _ok(load().pgm_graph_stats_get(g, C.byref(s)), "pgm_graph_stats_get")
    return {"n": s.n, "m": s.m, "dmax": s.dmax, "dag_dmax": s.dag_dmax,
            "sum_c2": int(s.sum_c2[0]) | (int(s.sum_c2[1]) << 64),
            "sum_c3": int(s.sum_c3[0]) | (int(s.sum_c3[1]) << 64)}


def pgm_graph_destroy(g: int):
    if g:
        load().pgm_graph_destroy(g)


# ---------------------------------------------------------------- counting
def pgm_count_kcliques(g: int, k: int) -> int:
    out = C.c_uint64()
    _ok(load().pgm_count_kcliques(g, k, C.byref(out)), "pgm_count_kcliques")
    return int(out.value)


def pgm_count_kcliques_range(g: int, k: int, v_lo: int, v_hi: int) -> int:
    out = C.c_uint64()
    _ok(load().pgm_count_kcliques_range(g, k, v_lo, v_hi, C.byref(out)), "pgm_count_kcliques_range")
    return int(out.value)


def pgm_list_kcliques(g: int, k: int, out_dev_ptr: int = 0, cap_rows: int = 0) -> int:
    """Rows of k vertex IDs (int32, row-major) into the device buffer at
    out_dev_ptr; returns the number of k-cliques (out_dev_ptr = 0: size query)."""
    n = C.c_int64()
    _ok(load().pgm_list_kcliques(g, k, out_dev_ptr or None, cap_rows, C.byref(n)), "pgm_list_kcliques")
    return int(n.value)


def pgm_list_kcliques_host(g: int, k: int, out=None) -> int:
    """Rows of k vertex IDs into the host array ``out`` (int32, shape (rows, k),
    C-contiguous; page-locked memory lets the copies overlap); returns the
    number of k-cliques (out = None: size query)."""
    n = C.c_int64()
    if out is None:
        _ok(load().pgm_list_kcliques_host(g, k, None, 0, C.byref(n)), "pgm_list_kcliques_host")
    else:
        if out.dtype != np.int32 or not out.flags["C_CONTIGUOUS"] or (out.ndim == 2 and out.shape[1] != k):
            raise ValueError("out must be a C-contiguous int32 array of shape (rows, k)")
        _ok(load().pgm_list_kcliques_host(g, k, out.ctypes.data, out.size // max(k, 1), C.byref(n)),
            "pgm_list_kcliques_host")
    return int(n.value)


def pgm_list_motifs(g: int, k: int, out_dev_ptr: int = 0, cap_rows: int = 0) -> int:
    """Rows of k vertex IDs (canonical order) + pattern index (int32, row-major,
    k + 1 per row) into the device buffer at out_dev_ptr; returns the number of
    connected k-sets (out_dev_ptr = 0: size query)."""
    n = C.c_int64()
    _ok(load().pgm_list_motifs(g, k, out_dev_ptr or None, cap_rows, C.byref(n)), "pgm_list_motifs")
    return int(n.value)


def pgm_list_motifs_host(g: int, k: int, out=None) -> int:
    """Rows of k vertex IDs (canonical order) + pattern index into the host
    array ``out`` (int32, shape (rows, k + 1), C-contiguous); returns the
    number of connected k-sets (out = None: size query)."""
    n = C.c_int64()
    if out is None:
        _ok(load().pgm_list_motifs_host(g, k, None, 0, C.byref(n)), "pgm_list_motifs_host")
    else:
        if out.dtype != np.int32 or not out.flags["C_CONTIGUOUS"] or (out.ndim == 2 and out.shape[1] != k + 1):
            raise ValueError("out must be a C-contiguous int32 array of shape (rows, k + 1)")
        _ok(load().pgm_list_motifs_host(g, k, out.ctypes.data, out.size // (k + 1), C.byref(n)),
            "pgm_list_motifs_host")
    return int(n.value)


def pgm_graph_set_labels(g: int, labels) -> None:
    """Vertex labels (int32 per vertex, each in [0, 2^15)) for pgm_fsm."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    _ok(load().pgm_graph_set_labels(g, lab.ctypes.data if lab.size else None), "pgm_graph_set_labels")


def pgm_fsm(g: int, max_edges: int, min_support: int = 1) -> list:
    """Frequent labelled patterns of 1..max_edges edges with MNI support >=
    min_support, as dicts {edges, labels (canonical order, tuple of nv),
    adj, support, embeddings} in the order (edges, nv, labels, adj)."""
    n = C.c_int32()
    cap = 1 << 16  # one mining run unless the result is larger (then a second with the exact size)
    buf = (pgm_fsm_pattern * cap)()
    rc = load().pgm_fsm(g, max_edges, min_support, buf, cap, C.byref(n))
    if rc == PGM_EOVERFLOW:
        cap = n.value
        buf = (pgm_fsm_pattern * cap)()
        rc = load().pgm_fsm(g, max_edges, min_support, buf, cap, C.byref(n))
    _ok(rc, "pgm_fsm")
    return [{"edges": p.edges, "labels": tuple(p.labels[:p.nv]), "adj": int(p.adj), "support": int(p.support),
             "embeddings": int(p.embeddings)} for p in buf[:n.value]]


def _npat(k: int) -> int:
    return {3: 2, 4: 6, 5: 21}.get(k, 0)


def pgm_count_motifs(g: int, k: int) -> list:
    out = np.zeros(21, np.uint64)
    _ok(load().pgm_count_motifs(g, k, out.ctypes.data, 21), "pgm_count_motifs")
    return [int(x) for x in out[: _npat(k)]]


def pgm_count_motifs_range(g: int, k: int, v_lo: int, v_hi: int) -> list:
    out = np.zeros(21, np.uint64)
    _ok(load().pgm_count_motifs_range(g, k, v_lo, v_hi, out.ctypes.data, 21), "pgm_count_motifs_range")
    return [int(x) for x in out[: _npat(k)]]


# ----------------------------------------------------------------- batches
def pgm_batch_create(G: int, vtx_off, rowptr_cat, col_cat, flags: int = 0, stream=None) -> int:
    vo = np.ascontiguousarray(vtx_off, dtype=np.int64)
    rp, cl = _host_csr(rowptr_cat, col_cat)
    h = P()
    _ok(load().pgm_batch_create(G, vo.ctypes.data, rp.ctypes.data, cl.ctypes.data, flags, _stream(stream),
                                C.byref(h)), "pgm_batch_create")
    return h.value


def _tune_ptr(t):
    return C.byref(t) if t is not None else None


def pgm_batch_count_motifs(b: int, k: int, tune: pgm_tune | None = None) -> np.ndarray:
    G = load().pgm_batch_size(b)
    out = np.zeros((max(G, 1), max(_npat(k), 1)), np.uint64)
    _ok(load().pgm_batch_count_motifs(b, k, out.ctypes.data, _tune_ptr(tune)), "pgm_batch_count_motifs")
    return out[:G]


def pgm_batch_count_kcliques(b: int, k: int, tune: pgm_tune | None = None) -> np.ndarray:
    G = load().pgm_batch_size(b)
    out = np.zeros(max(G, 1), np.uint64)
    _ok(load().pgm_batch_count_kcliques(b, k, out.ctypes.data, _tune_ptr(tune)), "pgm_batch_count_kcliques")
    return out[:G]


def pgm_batch_count_motifs_loop(b: int, k: int) -> np.ndarray:
    G = load().pgm_batch_size(b)
    out = np.zeros((max(G, 1), max(_npat(k), 1)), np.uint64)
    _ok(load().pgm_batch_count_motifs_loop(b, k, out.ctypes.data), "pgm_batch_count_motifs_loop")
    return out[:G]


def pgm_batch_autotune(b: int, k: int):
    t = pgm_tune()
    ms = C.c_double()
    _ok(load().pgm_batch_autotune(b, k, C.byref(t), C.byref(ms)), "pgm_batch_autotune")
    return t, float(ms.value)


def pgm_batch_autotune_ex(b: int, k: int, cache_path: str | None = None, cap: int = 64):
    """(best tune, best ms, [(tune dict, ms) per timed trial], came from the cache)."""
    t = pgm_tune()
    ms = C.c_double()
    tr = (pgm_tune_trial * max(cap, 1))()
    n = C.c_int32()
    hit = C.c_int32()
    path = cache_path.encode() if cache_path else None
    _ok(load().pgm_batch_autotune_ex(b, k, path, C.byref(t), C.byref(ms), tr, cap, C.byref(n), C.byref(hit)),
        "pgm_batch_autotune_ex")
    return t, float(ms.value), [(tr[i].tune.as_dict(), float(tr[i].ms)) for i in range(n.value)], bool(hit.value)


def pgm_batch_size(b: int) -> int:
    return int(load().pgm_batch_size(b))


def pgm_batch_destroy(b: int):
    if b:
        load().pgm_batch_destroy(b)


# ------------------------------------------------------------------ server
def pgm_server_create(budget_bytes: int, max_inflight: int) -> int:
    h = P()
    _ok(load().pgm_server_create(budget_bytes, max_inflight, C.byref(h)), "pgm_server_create")
    return h.value


def pgm_server_add_graph(s: int, n: int, rowptr, col) -> int:
    rp, cl = _host_csr(rowptr, col)
    gid = C.c_int32()
    _ok(load().pgm_server_add_graph(s, n, rp.ctypes.data, cl.ctypes.data, C.byref(gid)), "pgm_server_add_graph")
    return int(gid.value)


def pgm_server_submit(s: int, kind: int, k: int, graph: int) -> int:
    q = pgm_query(kind, k, graph, 0)
    t = C.c_int64()
    _ok(load().pgm_server_submit(s, C.byref(q), C.byref(t)), "pgm_server_submit")
    return int(t.value)


def pgm_server_poll(s: int, ticket: int) -> pgm_result:
    r = pgm_result()
    _ok(load().pgm_server_poll(s, ticket, C.byref(r)), "pgm_server_poll")
    return r


def pgm_server_drain(s: int, timeout_s: float):
    _ok(load().pgm_server_drain(s, timeout_s), "pgm_server_drain")


def pgm_server_destroy(s: int):
    if s:
        load().pgm_server_destroy(s)


# ----------------------------------------------------------- no allocation
def pgm_count_triangles_noalloc(n: int, dag_rowptr_dev_ptr: int, dag_col_dev_ptr: int, m: int,
                                count_dev_ptr: int, stream=None):
    """Triangle count of a caller-held device DAG, written to a caller-held
    device uint64, without any device allocation by the library."""
    _ok(load().pgm_count_triangles_noalloc(n, dag_rowptr_dev_ptr, dag_col_dev_ptr, m, count_dev_ptr,
                                           _stream(stream)), "pgm_count_triangles_noalloc")


# -------------------------------------------------------------------- misc
def pgm_set_options(**kw):
    o = pgm_options()
    for k, v in kw.items():
        setattr(o, k, v)
    _ok(load().pgm_set_options(C.byref(o)), "pgm_set_options")


def pgm_get_options() -> dict:
    o = pgm_options()
    _ok(load().pgm_get_options(C.byref(o)), "pgm_get_options")
    return {f: getattr(o, f) for f, _ in pgm_options._fields_ if f != "reserved"}


def pgm_debug_errors(reset: bool = False) -> int:
    """Out-of-range indices met by the bounds-checked build (always 0 otherwise)."""
    return int(load().pgm_debug_errors(1 if reset else 0))


def pgm_last_profile() -> dict:
    p = pgm_profile()
    _ok(load().pgm_last_profile(C.byref(p)), "pgm_last_profile")
    phases = []
    for i in range(p.nphases):
        ph = p.phase[i]
        phases.append({"name": ph.name.decode(), "level": ph.level, "launches": ph.launches, "ms": ph.ms,
                       "entries": ph.entries, "alg_bytes": ph.alg_bytes})
    return {"phases": phases, "level_size": [int(x) for x in p.level_size], "chunks": p.chunks}


def pgm_exclusive_scan_dev(cnt_dev_ptr: int, length: int, out_dev_ptr: int, stream=None):
    _ok(load().pgm_exclusive_scan_dev(cnt_dev_ptr, length, out_dev_ptr, _stream(stream)), "pgm_exclusive_scan_dev")


def pgm_last_error() -> str:
    return load().pgm_last_error().decode(errors="replace")


def pgm_version() -> str:
    return load().pgm_version().decode()


def pgm_kernel_launches() -> int:
    return int(load().pgm_kernel_launches())


# -------------------------------------------------------------- convenience
class Graph:
    """Owning wrapper of a pgm_graph handle (upload from a host CSR)."""

    def __init__(self, csr, flags: int = 0, stream=None):
        self.h = pgm_graph_create_csr(csr.n, csr.rowptr, csr.col, flags, stream)
        self.n = csr.n

    def orient(self):
        pgm_graph_orient_by_degree(self.h)
        return self

    def kcliques(self, k: int) -> int:
        return pgm_count_kcliques(self.h, k)

    def motifs(self, k: int) -> list:
        return pgm_count_motifs(self.h, k)

    def stats(self) -> dict:
        return pgm_graph_stats_get(self.h)

    def set_labels(self, labels):
        pgm_graph_set_labels(self.h, labels)
        return self

    def fsm(self, max_edges: int, min_support: int = 1) -> list:
        return pgm_fsm(self.h, max_edges, min_support)

    def close(self):
        if self.h:
            pgm_graph_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
