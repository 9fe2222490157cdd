"""NVTX ranges of the library, seen on the CPU through an NVTX injection
library (tests/nvtx_probe.c) instead of Nsight Systems: each public call
opens a range named after itself and closes it on every return path (here:
the argument-error paths, which need no GPU)."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import ctypes as C, sys
probe = C.CDLL(sys.argv[1])
from paper_1911_06969_b300 import pgm
L = pgm.load()
n = C.c_int32()
h = C.c_void_p()
calls = [
    ("pgm_graph_create_csr", L.pgm_graph_create_csr(-1, None, None, 0, None, C.byref(h))),
    ("pgm_fsm", L.pgm_fsm(None, 3, 1, None, 0, C.byref(n))),
    ("pgm_count_kcliques", L.pgm_count_kcliques(None, 4, None)),
    ("pgm_count_motifs", L.pgm_count_motifs(None, 4, None, 0)),
    ("pgm_graph_set_labels", L.pgm_graph_set_labels(None, None)),
]
assert all(rc == pgm.PGM_EINVAL for _, rc in calls), calls
probe.nvtx_probe_log.restype = C.c_char_p
print(probe.nvtx_probe_log().decode(), end="")
print("depth", probe.nvtx_probe_depth(), "max", probe.nvtx_probe_max_depth(), "pops", probe.nvtx_probe_pops())
"""


def nvtx_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "nvtx3", "nvToolsExt.h")) else None


def test_public_calls_open_and_close_named_ranges(tmp_path):
    inc = nvtx_include()
    if inc is None:
        pytest.skip("NVTX headers not found")
    lib = os.path.join(ROOT, "paper_1911_06969_b300", "libpgm.so")
    if not os.path.exists(lib):
        pytest.skip("libpgm.so not built")
    so = tmp_path / "libnvtx_probe.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-I", inc, "-o", str(so),
                           os.path.join(HERE, "nvtx_probe.c")])
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", CHILD, str(so)], env=env, capture_output=True, text=True,
                         cwd=ROOT, timeout=120)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().split("\n")
    assert lines[:5] == ["pgm_graph_create_csr", "pgm_fsm", "pgm_count_kcliques", "pgm_count_motifs",
                         "pgm_graph_set_labels"], lines
    assert lines[5] == "depth 0 max 1 pops 5"
