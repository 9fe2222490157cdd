"""The bounds-checked build (libpgm_debug.so, PGM_DEBUG): small cases of
every engine, with options that force the hub kernels, global-memory rows,
edge-blocking chunks and both 4-motif intersection variants, must give the
oracle's counts and meet no out-of-range index at the checked sites
(pgm_debug_errors() == 0).  Runs in a child process that loads the debug
library (PGM_LIB=debug); nothing traps in either build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import graphgen as gg, oracle
from paper_1911_06969_b300 import pgm
assert pgm.LIB_PATH.endswith("libpgm_debug.so"), pgm.LIB_PATH
pgm.pgm_debug_errors(True)
bad = []
settings = [dict(), dict(warp_stage_cap=32, hub_threshold=32, level_budget=1024, motif_b_side_min=1),
            dict(clique_engine=2, bitset_smem_degree=64, motif_b_side_min=1 << 30)]
graphs = [gg.barabasi_albert(1500, 7, seed=3), gg.rmat(1 << 11, 15000, seed=4), gg.chung_lu(4000, 2.1, 8.0, 400.0, 5)]
for st in settings:
    pgm.pgm_set_options(**st)
    for g in graphs:
        with pgm.Graph(g) as G:
            for k in (3, 4, 5, 7):
                if G.kcliques(k) != oracle.clique_count(g, k, "degree", threads=8):
                    bad.append((g.name, st, "clique", k))
            for k in (3, 4):
                if G.motifs(k) != oracle.formula_motifs(g, k, threads=8):
                    bad.append((g.name, st, "motif", k))
    g5 = gg.barabasi_albert(150, 3, seed=6)
    with pgm.Graph(g5) as G:
        if G.motifs(5) != oracle.esu_motifs(g5, 5):
            bad.append((g5.name, st, "motif", 5))
print(json.dumps({"bad": bad, "debug_errors": pgm.pgm_debug_errors(False),
                  "message": pgm.pgm_last_error() if pgm.pgm_debug_errors(False) else ""}))
"""


def test_debug_build_counts_and_no_bad_index():
    lib = os.path.join(ROOT, "paper_1911_06969_b300", "libpgm_debug.so")
    if not os.path.exists(lib):
        from paper_1911_06969_b300 import build

        build.build(debug=True)
    env = dict(os.environ, PGM_LIB="debug")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["bad"] == [], out
    assert out["debug_errors"] == 0, out["message"]
