"""GB300-native Domain Transform Solver (Bapat & Frahm, ECCV 2018).

The solver runs in hand-written CUDA kernels for sm_103a behind the C-ABI
library ``libdts.so`` (declared in ``include/dts.h``).  ``dts`` is the thin
Python binding with the same entry-point names; ``workloads`` draws the seeded
synthetic inputs.  Importing the package loads nothing: the CUDA library is
opened on first use, and every call fails loudly if it is missing.
"""
__all__ = ["dts", "workloads"]
