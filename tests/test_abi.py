"""The C ABI library loads on a machine without a GPU and exports every
function that include/pgm.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1911_06969_b300 import build, pgm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgm_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_header():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same names
    assert set(names) == set(pgm._SIGS), set(names) ^ set(pgm._SIGS)


def test_host_only_calls():
    lib = pgm.load()
    assert pgm.pgm_version().startswith("libpgm")
    o = pgm.pgm_get_options()
    assert o["block_threads"] == 256 and o["warp_stage_cap"] >= 32
    # argument validation happens before any device work
    import pytest

    with pytest.raises(pgm.PgmError) as e:
        pgm.pgm_set_options(block_threads=100)
    assert e.value.status == pgm.PGM_EINVAL
    with pytest.raises(pgm.PgmError):
        pgm.pgm_set_options(level_budget=5)
    assert lib.pgm_batch_size(None) == 0
    assert pgm.pgm_get_options()["block_threads"] == 256


def test_debug_library_exports_header():
    """The bounds-checked variant (PGM_DEBUG) exports the same ABI; without a
    device its error query reads no word and reports 0."""
    path = build.build(debug=True)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.pgm_debug_errors.restype = ctypes.c_uint64
    lib.pgm_debug_errors.argtypes = [ctypes.c_int32]
    assert lib.pgm_debug_errors(0) == 0
