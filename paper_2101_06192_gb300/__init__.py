"""Forest closeness centrality on GB300 (sm_103a): the UST-sampling estimator of
diag((I + alpha L)^{-1}) and the forest farness/closeness built on it.

The computation lives in libfc.so (CUDA, include/fc.h); this package is its
ctypes binding (``fc``) and in-tree build script (``build``).
"""
from . import build  # noqa: F401
