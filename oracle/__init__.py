"""ORACLE -- test infrastructure only.

A plain FP64 CPU implementation of the hydro update (C++, in this folder) and
an exact Riemann solver, wrapped with ctypes.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import this package; the CUDA
library never calls it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
