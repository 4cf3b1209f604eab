"""GB300-native swept time-space decomposition for 1D unsteady PDEs.

The compute path is the CUDA library ``libswept.so`` (sm_103a) behind the C ABI
declared in ``include/swept.h``; :mod:`paper_1705_03162_gb300.swept` is its
thin ctypes binding.  Importing this package loads nothing: the library is
loaded on first use and a missing library raises instead of falling back.
"""
__all__ = ["inputs", "swept"]
