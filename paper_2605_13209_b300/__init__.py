"""B300-native dense SPD solvers for Gaussian-process kernel systems.

The compute path is the CUDA library ``libgpchol.so`` (sources in ``csrc/``),
reached through its C ABI (``include/gpchol.h``) by the thin ctypes binding in
``gpchol.py``.  Importing this package does not load the library; the first
call into ``gpchol`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "gpchol"]
