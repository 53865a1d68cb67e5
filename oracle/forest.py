"""Forest roots and depths of sampled trees (test infrastructure only).

Removing u* from a spanning tree of G* rooted at u* leaves a rooted spanning
forest of G whose roots are the children of u* (Sec. 2: by the matrix-forest
theorem, Omega[u, v] is the weighted share of rooted spanning forests in which
v's tree is rooted at u).  For a parent array over V (parent[v] in 0..n, where
n stands for u*), the root of v is the vertex on v's path towards u* whose
parent is u*, and the depth of v is the number of edges from v to that root.
Both are read off by walking the parent pointers.
"""
from __future__ import annotations

import numpy as np


def roots_and_depths(parent) -> tuple[np.ndarray, np.ndarray]:
    """Per-vertex walk to u*: (root, depth), int64 [n].  Pure Python: small n."""
    parent = np.asarray(parent)
    n = parent.size
    root = np.empty(n, dtype=np.int64)
    depth = np.empty(n, dtype=np.int64)
    for v in range(n):
        x, d = v, 0
        while parent[x] != n:
            x = int(parent[x])
            d += 1
            if d > n:
                raise ValueError("parent pointers contain a cycle")
        root[v] = x
        depth[v] = d
    return root, depth


def roots_and_depths_np(parent) -> tuple[np.ndarray, np.ndarray]:
    """The same walk for every vertex at once, one parent step per round
    (rounds = the largest depth): (root, depth), int64 [n]."""
    parent = np.asarray(parent, dtype=np.int64)
    n = parent.size
    x = np.arange(n, dtype=np.int64)
    depth = np.zeros(n, dtype=np.int64)
    moving = parent != n
    for _ in range(n + 1):
        if not moving.any():
            return x, depth
        x[moving] = parent[x[moving]]
        depth[moving] += 1
        moving = parent[x] != n
    raise ValueError("parent pointers contain a cycle")
