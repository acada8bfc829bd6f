"""GB300-native construction of FMM data structures (arXiv:1301.1704).

The compute path lives in ``libfmmds.so`` (hand-written sm_103a CUDA behind a
C ABI, see ``include/fmmds.h``); :mod:`paper_1301_1704_gb300.fmmds` is the
ctypes binding.  Importing this package loads nothing; the binding raises if
the shared library has not been built.
"""

__all__ = ["fmmds", "workloads"]
