"""Rao-Blackwellised estimate of diag(Omega) from sampled trees (test
infrastructure only).

Prop. 1 estimates Omega[v, v] by the frequency with which v is joined to u*
in uniform spanning trees of G*.  Conditioning that indicator on the parents
of all other vertices leaves a smaller-variance unbiased estimate: with every
other parent fixed, the vertices whose path to u* runs through v (v's subtree
S(v), v included) are fixed, and v's parent can be u* (edge weight 1) or any
neighbour w outside S(v) (edge weight alpha * w_vw); each choice gives a
spanning tree whose weight is the same product times that edge's weight, so

    P(parent(v) = u* | the other parents)
        = 1 / (1 + alpha * sum over w in N(v) \\ S(v) of w_vw),

and the average of this over the sampled trees is unbiased for Omega[v, v]
(law of total expectation).  The sum runs over v's CSR row in order, in FP64
(weights converted from FP32), and the value is 1 / (1 + alpha * s) with
each operation rounded once.  Per tree the value is accumulated in fixed
point, q = floor(value * 2^48 + 1/2), so that totals do not depend on the
order in which trees are added; the estimate is sum(q) / (2^48 tau).

Everything here is a plain restatement: subtree membership by preorder
numbers and subtree sizes from an explicit depth-first traversal.
"""
from __future__ import annotations

import numpy as np

FRAC_BITS = 48


def subtree_intervals(parent: np.ndarray, n: int):
    """Preorder number tin[v] and subtree size size[v] of every vertex of the
    forest given by parent (parent[v] = n marks a root).  w lies in v's
    subtree iff tin[v] <= tin[w] < tin[v] + size[v]."""
    children = [[] for _ in range(n)]
    roots = []
    for v in range(n):
        p = int(parent[v])
        if p == n:
            roots.append(v)
        else:
            children[p].append(v)
    tin = np.empty(n, dtype=np.int64)
    size = np.ones(n, dtype=np.int64)
    clock = 0
    for r in roots:
        # iterative DFS: (vertex, next child index)
        stack = [(r, 0)]
        tin[r] = clock
        clock += 1
        while stack:
            v, i = stack[-1]
            if i < len(children[v]):
                stack[-1] = (v, i + 1)
                c = children[v][i]
                tin[c] = clock
                clock += 1
                stack.append((c, 0))
            else:
                stack.pop()
                if stack:
                    size[stack[-1][0]] += size[v]
    if clock != n:
        raise ValueError("parent array is not a spanning forest rooted at u*")
    return tin, size


def rb_values(g, alpha, parent: np.ndarray) -> np.ndarray:
    """P(parent(v) = u* | the other parents) for every vertex of one tree.
    alpha: a scalar or one value per vertex."""
    n = g.n
    tin, size = subtree_intervals(parent, n)
    av = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (n,))
    w = None if g.w is None else g.w.astype(np.float64)
    out = np.empty(n)
    for v in range(n):
        lo, hi = tin[v], tin[v] + size[v]
        s = 0.0
        for e in range(int(g.rowptr[v]), int(g.rowptr[v + 1])):
            t = tin[g.colidx[e]]
            if not (lo <= t < hi):
                s = s + (1.0 if w is None else float(w[e]))
        out[v] = 1.0 / (1.0 + float(av[v]) * s)
    return out


def to_fixed(values: np.ndarray) -> np.ndarray:
    """floor(value * 2^48 + 1/2) for values in [0, 1] (every step exact)."""
    return np.floor(values * float(1 << FRAC_BITS) + 0.5).astype(np.uint64)


def accumulate(g, alpha, parents: np.ndarray) -> np.ndarray:
    """Fixed-point sums over trees: parents has shape [tau, n]."""
    acc = np.zeros(g.n, dtype=np.uint64)
    for t in range(parents.shape[0]):
        acc += to_fixed(rb_values(g, alpha, parents[t]))
    return acc


def diag_from_fixed(acc: np.ndarray, tau: int) -> np.ndarray:
    return acc.astype(np.float64) / (float(1 << FRAC_BITS) * tau)
