"""Write the stored expected counts of the named workloads.

Calls only the CPU oracle (``oracle/``) and the input generators
(``graphgen/``); no value here comes from the CUDA library.  Run from the
repository root:

    python tests/golden/make_golden.py [triangle_er chung_lu_1m small_batch_20k serving_64 rmat21 rmat21_k5
                                        rmat_weak20 rmat_weak21 rmat_weak22]

Each workload writes ``tests/golden/<name>.json``.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))
THREADS = int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


def graph_digest(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.rowptr, np.int64).tobytes())
    h.update(np.ascontiguousarray(g.col, np.int32).tobytes())
    return h.hexdigest()


def write(name, d):
    with open(os.path.join(OUT, f"{name}.json"), "w") as f:
        json.dump(d, f, indent=1)
    print(name, json.dumps(d)[:400], flush=True)


def stats(g):
    s2, s3, dmax = oracle.degree_sums(g)
    return {"n": g.n, "m": g.m, "dmax": dmax, "sum_C_d_2": s2, "sum_C_d_3": s3}


def do_triangle_er():
    g = gg.triangle_er()
    t = time.time()
    d = {"workload": "Erdos-Renyi n=4096, p=16/4095, seed 1", "graph_sha256": graph_digest(g), **stats(g),
         "clique_levels_k7": oracle.clique_levels(g, 7, "id", threads=THREADS),
         "motif3": oracle.esu_motifs(g, 3), "motif4": oracle.esu_motifs(g, 4),
         "motif4_formula": oracle.formula_motifs(g, 4)}
    d["oracle_seconds"] = round(time.time() - t, 2)
    write("triangle_er", d)


def _rmat21(k, name):
    g = gg.rmat21()
    t = time.time()
    lv = oracle.clique_levels(g, k, "degree", threads=THREADS)
    d = {"workload": "R-MAT scale 21, (a,b,c,d)=(0.57,0.19,0.19,0.05), 28,000,000 edges, seed 1",
         "graph_sha256": graph_digest(g), **stats(g), f"clique_levels_k{k}": lv,
         "oracle": "orc_clique_count, (degree, ID) order", "oracle_threads": THREADS,
         "oracle_seconds": round(time.time() - t, 1)}
    write(name, d)


def do_rmat21():
    _rmat21(4, "rmat21")


def do_rmat21_k5():
    _rmat21(5, "rmat21_k5")


def do_chung_lu_1m():
    g = gg.chung_lu_1m()
    t = time.time()
    m3 = oracle.formula_motifs(g, 3, threads=THREADS)
    m4 = oracle.formula_motifs(g, 4, threads=THREADS)
    d = {"workload": "Chung-Lu n=2^20, exponent 2.1, mean weight 10, weight cap 20000, seed 1",
         "graph_sha256": graph_digest(g), **stats(g), "motif3": m3, "motif4": m4,
         "oracle": "orc_formula_motifs", "oracle_threads": THREADS,
         "oracle_seconds": round(time.time() - t, 1)}
    write("chung_lu_1m", d)


def do_small_batch_20k():
    b = gg.small_batch_20k()
    t = time.time()
    m4 = oracle.formula_motifs_batch(b, 4)
    m3 = oracle.formula_motifs_batch(b, 3)
    d = {"workload": "20,000 graphs, n in [16,4096], even ER (degree 4-32), odd BA (m 2-8), seed 1",
         "graph_sha256": graph_digest(b.graph), "G": b.G, "n": b.graph.n, "arcs": b.graph.narcs,
         "motif4_sha256": hashlib.sha256(np.ascontiguousarray(m4, np.uint64).tobytes()).hexdigest(),
         "motif3_sha256": hashlib.sha256(np.ascontiguousarray(m3, np.uint64).tobytes()).hexdigest(),
         "motif4_total": [int(x) for x in m4.astype(object).sum(0)],
         "motif3_total": [int(x) for x in m3.astype(object).sum(0)],
         "motif4_first64": [[int(x) for x in r] for r in m4[:64]],
         "motif3_first64": [[int(x) for x in r] for r in m3[:64]],
         "oracle": "orc_formula_motifs_batch", "oracle_seconds": round(time.time() - t, 1)}
    write("small_batch_20k", d)


def do_serving_64():
    b = gg.serving_64()
    t = time.time()
    rows = []
    for i in range(b.G):
        g = b.part(i)
        lv = oracle.clique_levels(g, 4, "degree", threads=THREADS)
        rows.append({"n": g.n, "m": g.m, "kind": int(b.kind[i]), "triangles": lv[3], "k4": lv[4],
                     "motif3": oracle.formula_motifs(g, 3, threads=THREADS)})
    d = {"workload": "64 resident graphs: 32 R-MAT + 32 BA, n log-uniform [1e3,1e6], degree 8-32, seed 1",
         "graph_sha256": graph_digest(b.graph), "G": b.G, "graphs": rows,
         "oracle_seconds": round(time.time() - t, 1)}
    write("serving_64", d)


def _rmat_weak(scale):
    g = gg.rmat_weak(scale)
    t = time.time()
    lv = oracle.clique_levels(g, 4, "degree", threads=THREADS)
    d = {"workload": f"R-MAT scale {scale}, (a,b,c,d)=(0.57,0.19,0.19,0.05), average degree 20 "
                     f"({10 << scale:,} edges), seed 1",
         "graph_sha256": graph_digest(g), **stats(g), "clique_levels_k4": lv,
         "motif3": oracle.formula_motifs(g, 3, threads=THREADS),
         "oracle": "orc_clique_count, (degree, ID) order; orc_formula_motifs", "oracle_threads": THREADS,
         "oracle_seconds": round(time.time() - t, 1)}
    write(f"rmat_weak{scale}", d)


def do_rmat_weak20():
    _rmat_weak(20)


def do_rmat_weak21():
    _rmat_weak(21)


def do_rmat_weak22():
    _rmat_weak(22)


if __name__ == "__main__":
    names = sys.argv[1:] or ["triangle_er", "chung_lu_1m", "small_batch_20k", "serving_64", "rmat21", "rmat21_k5"]
    for nm in names:
        globals()[f"do_{nm}"]()
