"""Brute-force enumeration of the spanning trees of G* (test infrastructure only).

A spanning tree of G* is the same object as a spanning rooted forest of G (cut
the edges at u*; the vertices that were joined to u* are the roots).  Weighting
each tree by the product of its edge weights in G* (alpha w_e for edges of G,
1 for edges to u*), the matrix-forest theorem (Sec. 2: Omega[u, v] is the share
of rooted spanning forests in which u and v lie in one tree; the share is
weighted in the weighted case, Prop. 1 proof) gives

    Omega[u, v] = (total weight of trees in which the path from v to u*
                   enters u* through u) / (total weight of all trees),

and Kirchhoff's theorem gives total weight = det(I + alpha L).  Only for tiny
graphs (|E| + n <= ~22).
"""
from __future__ import annotations

import itertools

import numpy as np


def augmented_edges(g, alpha: float):
    """Edge list of G*: (u, v, weight), u* = n."""
    u, v, w = g.edges()
    w = np.ones(u.size) if w is None else w.astype(np.float64)
    edges = [(int(a), int(b), float(alpha * c)) for a, b, c in zip(u, v, w)]
    edges += [(i, g.n, 1.0) for i in range(g.n)]
    return edges


def spanning_trees(g, alpha: float):
    """Yield (parent array of length n rooted at u* = n, weight) for every
    spanning tree of G*."""
    n = g.n
    E = augmented_edges(g, alpha)
    for subset in itertools.combinations(range(len(E)), n):
        parent_uf = list(range(n + 1))

        def find(x):
            while parent_uf[x] != x:
                parent_uf[x] = parent_uf[parent_uf[x]]
                x = parent_uf[x]
            return x

        ok = True
        weight = 1.0
        adj = [[] for _ in range(n + 1)]
        for ei in subset:
            a, b, c = E[ei]
            ra, rb = find(a), find(b)
            if ra == rb:
                ok = False
                break
            parent_uf[ra] = rb
            weight *= c
            adj[a].append(b)
            adj[b].append(a)
        if not ok:
            continue
        # orient towards u* by BFS from u*
        par = [-2] * (n + 1)
        par[n] = -1
        stack = [n]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if par[y] == -2:
                    par[y] = x
                    stack.append(y)
        yield np.array(par[:n], dtype=np.int32), weight


def tree_distribution(g, alpha: float):
    """dict: parent-array bytes -> probability (weight / total weight), and the
    total weight."""
    dist = {}
    total = 0.0
    for par, wt in spanning_trees(g, alpha):
        dist[par.tobytes()] = wt
        total += wt
    return {k: v / total for k, v in dist.items()}, total


def omega_by_forests(g, alpha: float) -> np.ndarray:
    """Omega from the matrix-forest theorem: Omega[u, v] = P(v's path to u*
    enters u* through u)."""
    n = g.n
    num = np.zeros((n, n))
    total = 0.0
    for par, wt in spanning_trees(g, alpha):
        total += wt
        for v in range(n):
            x = v
            while par[x] != n:
                x = par[x]
            num[x, v] += wt
    return num / total
