"""Group forest closeness (Sec. 5, Algorithm 3): test infrastructure only,
never called by the product path.

Definitions, written out with numpy primitives:
  * group forest farness rho(S) = tr((L*_{-S})^{-1}), where L* is the
    Laplacian of the augmented graph G* (Sec. 4.1; `dense.augmented_laplacian`)
    and L*_{-S} drops the rows and columns of the vertices in S (u* stays);
    group forest closeness is 1 / rho(S);
  * the greedy maximiser of Algorithm 3: start from the vertex minimising
    n L*^+[v, v] + tr(L*^+) (the vertex of highest individual forest
    closeness), keep M = (L*_{-S})^{-1}, add the vertex v of V \\ S (never
    u*) maximising ||M e_v||^2 / (e_v^T M e_v), and update M by the rank-one
    downdate M - M e_v e_v^T M / (e_v^T M e_v) restricted to the remaining
    indices.

Readings: Algorithm 3's loop condition |S| <= k would return k + 1 vertices
while its output is a group of k vertices; the loop here runs while |S| < k.
Ties in the argmin / argmax go to the smallest vertex id.
"""
from __future__ import annotations

import numpy as np

from . import dense


def group_farness(g, alpha: float, S) -> float:
    """rho(S) = tr((L*_{-S})^{-1}) by a dense inverse (the definition)."""
    Ls = dense.augmented_laplacian(g, alpha)
    keep = np.setdiff1d(np.arange(g.n + 1), np.asarray(list(S), dtype=np.int64))
    return float(np.trace(np.linalg.inv(Ls[np.ix_(keep, keep)])))


def greedy(g, alpha: float, k: int, with_gains: bool = False):
    """Algorithm 3.  Returns (S, farness) with S the chosen vertices in order
    and farness[i] = rho(S[:i+1]) read off the maintained inverse; with
    with_gains, also the gain of every candidate at every step (dicts)."""
    n = g.n
    if not 1 <= k <= n:
        raise ValueError("need 1 <= k <= n")
    Ls = dense.augmented_laplacian(g, alpha)
    P = np.linalg.pinv(Ls)
    score = n * np.diag(P)[:n] + np.trace(P)
    v = int(np.argmin(score))  # first occurrence: smallest id among ties
    idx = [i for i in range(n + 1) if i != v]  # rows / columns of M, in order
    M = np.linalg.inv(Ls[np.ix_(idx, idx)])
    S = [v]
    far = [float(np.trace(M))]
    all_gains = []
    while len(S) < k:
        best, bj = -np.inf, -1
        step = {}
        for j, vert in enumerate(idx):
            if vert == n:  # u* is never chosen
                continue
            col = M[:, j]
            gain = float(col @ col) / float(M[j, j])
            step[vert] = gain
            if gain > best:
                best, bj = gain, j
        all_gains.append(step)
        col = M[:, bj].copy()
        M = M - np.outer(col, col) / col[bj]
        M = np.delete(np.delete(M, bj, axis=0), bj, axis=1)
        S.append(idx[bj])
        del idx[bj]
        far.append(float(np.trace(M)))
    if with_gains:
        return S, np.array(far), all_gains
    return S, np.array(far)


def gains(g, alpha: float, S):
    """Marginal gains rho(S) - rho(S + {v}) for every v of V \\ S, each from
    two dense inverses (the definition; used to check the greedy choice)."""
    base = group_farness(g, alpha, S)
    out = {}
    for v in range(g.n):
        if v in S:
            continue
        out[v] = base - group_farness(g, alpha, list(S) + [v])
    return out
