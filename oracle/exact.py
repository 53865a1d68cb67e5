"""Exact rational arithmetic for tiny graphs (test infrastructure only).

Omega = (alpha L + I)^{-1} (Sec. 2) by Gauss-Jordan elimination over Python
Fractions, and the same matrix from the matrix-forest theorem (Sec. 2, Omega[u,v]
is the weighted share of rooted spanning forests in which u and v share a tree)
by enumerating spanning trees of G* with Fraction weights.  Used to write the
golden fixtures in tests/golden/ and to pin the FP64 routines.
"""
from __future__ import annotations

import itertools
from fractions import Fraction


def omega_gauss_jordan(n: int, edges, alpha: Fraction):
    """edges: list of (u, v, w) with Fraction w.  Returns Omega as nested lists."""
    M = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        M[i][i] = Fraction(1)
    for u, v, w in edges:
        M[u][u] += alpha * w
        M[v][v] += alpha * w
        M[u][v] -= alpha * w
        M[v][u] -= alpha * w
    A = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [row[n:] for row in A]


def omega_forests(n: int, edges, alpha: Fraction):
    """Omega from spanning trees of G* (u* = n) with exact weights; also returns
    the total tree weight, which equals det(I + alpha L) (Kirchhoff)."""
    E = [(u, v, alpha * w) for u, v, w in edges] + [(i, n, Fraction(1)) for i in range(n)]
    num = [[Fraction(0)] * n for _ in range(n)]
    total = Fraction(0)
    for subset in itertools.combinations(range(len(E)), n):
        uf = list(range(n + 1))

        def find(x):
            while uf[x] != x:
                uf[x] = uf[uf[x]]
                x = uf[x]
            return x

        ok = True
        wt = Fraction(1)
        adj = [[] for _ in range(n + 1)]
        for ei in subset:
            a, b, c = E[ei]
            ra, rb = find(a), find(b)
            if ra == rb:
                ok = False
                break
            uf[ra] = rb
            wt *= c
            adj[a].append(b)
            adj[b].append(a)
        if not ok:
            continue
        par = [-2] * (n + 1)
        par[n] = -1
        st = [n]
        while st:
            x = st.pop()
            for y in adj[x]:
                if par[y] == -2:
                    par[y] = x
                    st.append(y)
        total += wt
        for v in range(n):
            x = v
            while par[x] != n:
                x = par[x]
            num[x][v] += wt
    return [[x / total for x in row] for row in num], total


def _inverse(M):
    """Exact inverse of a nonsingular Fraction matrix by Gauss-Jordan."""
    k = len(M)
    A = [row[:] + [Fraction(int(i == j)) for j in range(k)] for i, row in enumerate(M)]
    for col in range(k):
        piv = next(r for r in range(col, k) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(k):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [row[k:] for row in A]


def group_farness(n: int, edges, alpha: Fraction, S):
    """rho(S) = tr((L*_{-S})^{-1}) (Sec. 5) exactly: L* is the Laplacian of
    G* (edges of G scaled by alpha, every vertex joined to u* = n by weight 1)
    with the rows and columns of S removed."""
    L = [[Fraction(0)] * (n + 1) for _ in range(n + 1)]
    for u, v, w in edges:
        L[u][u] += alpha * w
        L[v][v] += alpha * w
        L[u][v] -= alpha * w
        L[v][u] -= alpha * w
    for v in range(n):
        L[v][v] += 1
        L[n][n] += 1
        L[v][n] -= 1
        L[n][v] -= 1
    keep = [i for i in range(n + 1) if i not in set(S)]
    inv = _inverse([[L[i][j] for j in keep] for i in keep])
    return sum(inv[i][i] for i in range(len(keep)))
