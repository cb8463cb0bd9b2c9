"""GB300-native (sm_103a) evaluation of the frequency-domain Whittle log-likelihood of
massive-black-hole-binary signals for LISA-, Taiji- and TianQin-like detectors
(arXiv:2602.12011, pespace).

The compute path is the C-ABI library libpespace_gb300.so (include/pespace_gb300.h), built
in-tree by paper_2602_12011_gb300.build; ``_lib`` is its ctypes binding. Importing the package
loads nothing; the first library call raises if the library is missing (no CPU fallback).
"""
from . import workloads  # noqa: F401  (inputs only: no method arithmetic)

__all__ = ["workloads"]
