"""ctypes loader for the oracle's C sampler (test infrastructure only).

``build()`` compiles ``wilson_oracle.c`` with gcc (-O2 -ffp-contract=off, no
target-specific flags, so x86_64 and aarch64 give identical results).  Every
function here runs single-threaded; ctypes releases the GIL during the call, so
callers may run several tree ranges in parallel threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.orc_wilson.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_double, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P]
        L.orc_wilson.restype = ctypes.c_int
        L.orc_wilson_v.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_double, P, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P]
        L.orc_wilson_v.restype = ctypes.c_int
        L.orc_philox_batch.argtypes = [ctypes.c_int64, P, ctypes.c_uint64, P]
        L.orc_philox_batch.restype = None
        L.orc_row_prefix.argtypes = [ctypes.c_int32, P, P, P]
        L.orc_row_prefix.restype = None
        L.orc_p_root.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_p_root.restype = ctypes.c_double
        L.orc_stack_entries.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_double, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, P, P, P]
        L.orc_stack_entries.restype = ctypes.c_int
        L.orc_wilson_rooted.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_int64, P, P, P, P]
        L.orc_wilson_rooted.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox(ctrs: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 of each counter row (uint32[k, 4]) under key (seed_lo, seed_hi)."""
    ctrs = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctrs)
    lib().orc_philox_batch(ctrs.shape[0], _ptr(ctrs), int(seed) & (2**64 - 1), _ptr(out))
    return out


def row_prefix(g) -> np.ndarray:
    S = np.zeros(max(g.nnz, 1), dtype=np.float64)
    lib().orc_row_prefix(g.n, _ptr(g.rowptr), _ptr(np.ascontiguousarray(g.w, np.float32)), _ptr(S))
    return S[: g.nnz]


def p_root(d: int, alpha: float, S_d: float, weighted: bool) -> float:
    return float(lib().orc_p_root(int(d), float(alpha), float(S_d), int(bool(weighted))))


def stack_entries(g, alpha: float, seed: int, tree: int, verts, ks, alpha_idx: int = 0):
    """Vertex chosen by stack entry ks[i] of verts[i] in tree ``tree`` (n = u*)."""
    verts = np.ascontiguousarray(verts, dtype=np.int32)
    ks = np.ascontiguousarray(ks, dtype=np.uint32)
    out = np.empty(verts.size, dtype=np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)
    rc = lib().orc_stack_entries(g.n, _ptr(g.rowptr), _ptr(g.colidx), _ptr(w), float(alpha),
                                 int(alpha_idx), int(seed) & (2**64 - 1), int(tree), verts.size,
                                 _ptr(verts), _ptr(ks), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def wilson(g, alpha, seed: int, tau: int, tree_offset: int = 0, alpha_idx: int = 0,
           order=None, want_parents: bool = False, want_C: bool = True, want_steps: bool = True,
           want_visits: bool = False):
    """Sequential Wilson sampler on G* (Algorithm 2).  ``alpha`` is a float or a
    per-vertex array (a batch of graphs as one block-diagonal union).  Returns
    dict with R, C, parents ([tau, n], n = u*), steps ([tau]) and visits ([n],
    departures from each vertex summed over the trees)."""
    n = g.n
    R = np.zeros(n, dtype=np.uint32)
    C = np.zeros(n, dtype=np.uint32) if want_C else None
    parents = np.empty((tau, n), dtype=np.int32) if want_parents else None
    steps = np.zeros(tau, dtype=np.uint64) if want_steps else None
    visits = np.zeros(n, dtype=np.uint64) if want_visits else None
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)
    order_arr = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    av = None
    if np.ndim(alpha) > 0:
        av = np.ascontiguousarray(alpha, dtype=np.float64)
        assert av.size == n
        alpha = 0.0
    rc = lib().orc_wilson_v(n, _ptr(g.rowptr), _ptr(g.colidx), _ptr(w), float(alpha), _ptr(av), int(alpha_idx),
                            int(seed) & (2**64 - 1), int(tree_offset), int(tau), _ptr(order_arr),
                            _ptr(R), _ptr(C), _ptr(parents), _ptr(steps), _ptr(visits))
    if rc != 0:
        raise MemoryError("oracle sampler allocation failed")
    return {"R": R, "C": C, "parents": parents, "steps": steps, "visits": visits}


def wilson_rooted(g, root: int, seed: int, tau: int, tree_offset: int = 0, order=None,
                  want_parents: bool = True, want_steps: bool = True, want_visits: bool = False):
    """Sequential Wilson sampler on G rooted at ``root`` (uniform spanning trees
    of G, walks with probability w_vj / d_w(v)).  Returns dict with parents
    ([tau, n], the root's entry n), steps ([tau], departures) and visits ([n],
    departures from each vertex summed over the trees; the root's 0)."""
    n = g.n
    parents = np.empty((tau, n), dtype=np.int32) if want_parents else None
    steps = np.zeros(tau, dtype=np.uint64) if want_steps else None
    visits = np.zeros(n, dtype=np.uint64) if want_visits else None
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)
    order_arr = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    rc = lib().orc_wilson_rooted(n, _ptr(g.rowptr), _ptr(g.colidx), _ptr(w), int(root), int(seed) & (2**64 - 1),
                                 int(tree_offset), int(tau), _ptr(order_arr), _ptr(parents), _ptr(steps),
                                 _ptr(visits))
    if rc == -2:
        raise ValueError("wilson_rooted: the graph is not connected")
    if rc != 0:
        raise MemoryError("oracle sampler allocation failed")
    return {"parents": parents, "steps": steps, "visits": visits}
