"""GB300 (sm_103a) implementation of the CAC-MFZ-CDP compressed-sensing solver.

The compute path is libcs.so (CUDA kernels behind the C ABI of include/cs.h);
``paper_2405_00366_gb300.cs`` is its ctypes binding with the same names.  The
library is loaded on first use and its absence is an error.
"""
from . import build, cs  # noqa: F401

__all__ = ["build", "cs"]
