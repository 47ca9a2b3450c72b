"""GB300-native convolution gridding (the data-parallel hot path of HEGrid).

The compute path lives in ``libhegrid.so`` (hand-written CUDA for sm_103a
behind a C ABI, ``include/hegrid.h``); :mod:`.hegrid` is a thin ctypes binding
with the same names.  Importing this package does not load the library; the
first call into :mod:`.hegrid` does, and fails loudly if it is missing.
"""
__all__ = ["hegrid", "workloads"]
