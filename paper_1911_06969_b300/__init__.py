"""B300-native (sm_103a) exact k-clique and k-motif counting with the
extend-reduce model of Pangolin (level-wise embedding lists, connectivity
checks by sorted intersection / binary search, customised pattern
classification, count reduction).

The compute path is ``libpgm.so`` (CUDA, built from ``csrc/`` by
``build.py``), whose C ABI is ``include/pgm.h``; ``pgm`` is its ctypes
binding.
"""
from . import pgm  # noqa: F401
from .pgm import Graph, PgmError  # noqa: F401
