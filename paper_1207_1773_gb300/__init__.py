"""gbhegv: GB300-native two-stage Hermitian-definite generalized eigensolver.

The compute path lives in the CUDA library ``libgbhegv.so`` (C-ABI declared
in ``include/gbhegv.h``); ``paper_1207_1773_gb300.gbhegv`` is the thin ctypes
binding.  Importing this package does not load the library; the binding does,
and fails loudly if it is missing.
"""
__all__ = ["inputs"]
