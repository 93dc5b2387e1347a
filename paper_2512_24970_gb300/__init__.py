"""GB300-native RBSOG + RBL force evaluation and MD step for BMH ionic systems.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI in
``include/rbsog.h``); :mod:`paper_2512_24970_gb300.rbsog` is its thin ctypes
binding and :mod:`paper_2512_24970_gb300.workloads` builds seeded inputs.
Importing the package loads nothing; the library is loaded on first use and
its absence is an error (there is no CPU fallback).
"""
__all__ = ["rbsog", "workloads"]
