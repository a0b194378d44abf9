"""GB300-native frozen Gaussian approximation (FGA) for the 3-D elastic wave equation.

The compute path is the C-ABI library ``libfga_gb300.so`` (hand-written sm_103a CUDA, declared
in ``include/fga.h``); ``paper_1810_06760_gb300.fga`` is the thin ctypes binding with the same
entry-point names.  Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["fga", "workloads", "build"]
