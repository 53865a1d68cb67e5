"""Electrical closeness on G and its UST estimator (test infrastructure only).

The paper builds on an algorithm for diag(L^+) of a connected graph G (Sec. 3,
the proposition quoted from Angriman et al. and its three insights), which the
forest algorithm transfers to G*.  What it computes, from the definitions:

  * L^+, the Moore-Penrose pseudo-inverse of the Laplacian L of G (Sec. 2);
  * effective resistance r(u, v) = L^+[u,u] + L^+[v,v] - 2 L^+[u,v]  (Eq. 2);
  * electrical farness and closeness: Def. 2 with the forest distance
    replaced by r (Sec. 2): far(u) = sum_{v != u} r(u, v) = n L^+[u,u] +
    tr(L^+) (the rows of L^+ sum to zero), closeness(u) = n / far(u).

The estimator follows the three insights: (ii) one Laplacian solve gives the
pivot column x = L^+ e_u, and Eq. 2 turns r(u, v) for all v into
    L^+[v, v] = r(u, v) - x[u] + 2 x[v];
(iii) r(u, v) is estimated from uniform spanning trees of G.  For an edge
{u, v} the paper states it as r = P({u, v} in T) (weighted: / w_uv,
Kirchhoff); for non-adjacent pairs the paper leaves the aggregation along
shortest paths to the cited work, so it is restated here from Kirchhoff's
current theorem: in a UST T the tree path from v to u crosses the directed
edge a -> b with probability P(a->b) and a unit current sent from v to u
puts current P(a->b) - P(b->a) on {a, b}.  Summing the potential drops
current / w along ANY fixed path from v to u gives r(u, v); with T rooted at
u (every vertex points to its tree parent, the path from v to u is v's chain
of ancestors) and the fixed path taken from a breadth-first tree B of u,
    S_T(v) = sum over the edges (x, b(x)) of v's B-path, from v upward, of
             ( [par_T(x) = b(x) and x is an ancestor-or-self of v in T]
             - [par_T(b(x)) = x and b(x) is an ancestor-or-self of v in T] ) / w(x, b(x))
is unbiased for r(u, v).  (Pinned below by exact expectation over all
spanning trees of small graphs, not by this derivation.)

Readings: B is the breadth-first tree of u in which the parent of v is its
smallest-id neighbour one level closer to u.  S_T(v) is summed in FP64 in
path order, s = s + c * (1 / w) with c in {-1, 0, +1} and 1 / w one FP64
division of the FP32 weight converted to FP64 (1 for unweighted graphs); per
tree it enters a signed fixed-point total floor(S_T(v) * 2^32 + 1/2), so
totals do not depend on the order of the trees; r^ = total / (2^32 tau).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import dense

FRAC_BITS = 32


# ---- definitions ------------------------------------------------------------
def is_connected(g) -> bool:
    return bool(np.all(bfs_tree(g, 0)[1] >= 0)) if g.n > 0 else True


def laplacian_pinv(g) -> np.ndarray:
    """L^+ of a connected graph: (L + J/n)^{-1} - J/n (L has kernel span(1))."""
    if not is_connected(g):
        raise ValueError("laplacian_pinv: G must be connected")
    n = g.n
    L = dense.laplacian(g)
    J = np.full((n, n), 1.0 / n)
    return np.linalg.inv(L + J) - J


def resistance(Lp: np.ndarray, u: int, v: int) -> float:
    """Eq. 2."""
    return float(Lp[u, u] + Lp[v, v] - 2.0 * Lp[u, v])


def resistance_matrix(Lp: np.ndarray) -> np.ndarray:
    d = np.diag(Lp)
    return d[:, None] + d[None, :] - 2.0 * Lp


def electrical_farness(Lp: np.ndarray) -> np.ndarray:
    """sum over v != u of r(u, v), written out from Eq. 2."""
    return resistance_matrix(Lp).sum(axis=1)


def electrical_closeness(farness: np.ndarray) -> np.ndarray:
    """Def. 2 with r in place of the forest distance: n / farness."""
    return farness.size / farness


# ---- the breadth-first tree of the pivot -------------------------------------
def bfs_tree(g, root: int):
    """(parent, depth): breadth-first levels from root; the parent of v != root
    is its smallest-id neighbour one level closer (root: -1; unreachable
    vertices: parent -1 and depth -1).  Frontiers as numpy arrays."""
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr))
    dst = g.colidx.astype(np.int64)
    depth = np.full(n, -1, dtype=np.int64)
    depth[root] = 0
    frontier = np.array([root], dtype=np.int64)
    level = 0
    while frontier.size:
        # every neighbour of the frontier not yet reached joins the next level
        rows = [dst[g.rowptr[x]:g.rowptr[x + 1]] for x in frontier] if frontier.size < 64 else None
        nb = np.concatenate(rows) if rows is not None else dst[np.isin(src, frontier)]
        nb = np.unique(nb[depth[nb] < 0])
        level += 1
        depth[nb] = level
        frontier = nb
    parent = np.full(n, -1, dtype=np.int64)
    closer = (depth[src] > 0) & (depth[dst] == depth[src] - 1)
    big = np.iinfo(np.int64).max
    best = np.full(n, big, dtype=np.int64)
    np.minimum.at(best, src[closer], dst[closer])
    has = best != big
    parent[has] = best[has]
    return parent, depth


def edge_weight(g, a: int, b: int) -> float:
    for e in range(g.rowptr[a], g.rowptr[a + 1]):
        if int(g.colidx[e]) == b:
            return 1.0 if g.w is None else float(g.w[e])
    raise KeyError((a, b))


def bfs_inverse_weights(g, bpar) -> np.ndarray:
    """1 / w(v, b(v)) in FP64 (0 for the root), one FP64 division of the FP32
    weight converted to FP64 (1 for unweighted graphs)."""
    bpar = np.asarray(bpar, dtype=np.int64)
    inv = np.zeros(g.n)
    has = bpar >= 0
    if g.w is None:
        inv[has] = 1.0
        return inv
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    hit = g.colidx.astype(np.int64) == bpar[src]  # the CSR entry (v, b(v)) of each row
    inv[src[hit]] = 1.0 / g.w[hit].astype(np.float64)
    return inv


# ---- the per-tree path sums ---------------------------------------------------
def tree_intervals(parent: np.ndarray, root: int):
    """Preorder numbers and subtree sizes of the tree given by parent (parent of
    the root: anything outside [0, n)); a is an ancestor-or-self of v iff
    tin[a] <= tin[v] < tin[a] + size[a]."""
    n = parent.size
    children = [[] for _ in range(n)]
    for v in range(n):
        if v != root:
            children[int(parent[v])].append(v)
    tin = np.zeros(n, dtype=np.int64)
    size = np.ones(n, dtype=np.int64)
    order = []
    stack = [root]
    while stack:
        x = stack.pop()
        tin[x] = len(order)
        order.append(x)
        stack.extend(reversed(children[x]))
    for x in reversed(order):
        if x != root:
            size[int(parent[x])] += size[x]
    return tin, size


def path_sums(g, root: int, bpar, binv, parent: np.ndarray) -> np.ndarray:
    """S_T(v) for every v for one tree T (parent array rooted at root)."""
    n = g.n
    tin, size = tree_intervals(parent, root)

    def anc(a, v):
        return tin[a] <= tin[v] < tin[a] + size[a]

    out = np.zeros(n)
    for v in range(n):
        s = 0.0
        x = v
        while x != root:
            b = int(bpar[x])
            c = 0
            if int(parent[x]) == b and anc(x, v):
                c += 1
            if b != root and int(parent[b]) == x and anc(b, v):
                c -= 1
            if c != 0:
                s = s + c * binv[x]
            x = b
        out[v] = s
    return out


def path_sums_np(g, root: int, bpar, binv, parent: np.ndarray) -> np.ndarray:
    """path_sums with the walk along the BFS paths taken for all vertices at
    once (numpy, same FP64 additions in the same order per vertex; a zero
    term leaves s unchanged exactly).  For large graphs."""
    n = g.n
    tin, size = tree_intervals(parent, root)
    bpar = np.asarray(bpar, dtype=np.int64)
    parent = np.asarray(parent, dtype=np.int64)
    tv = tin
    x = np.arange(n, dtype=np.int64)
    s = np.zeros(n)
    live = x != root
    while live.any():
        xs = x[live]
        b = bpar[xs]
        tvl = tv[live]
        up = (parent[xs] == b) & (tin[xs] <= tvl) & (tvl < tin[xs] + size[xs])
        bb = np.where(b == root, 0, b)
        down = (b != root) & (parent[bb] == xs) & (tin[bb] <= tvl) & (tvl < tin[bb] + size[bb])
        c = up.astype(np.float64) - down.astype(np.float64)
        s[live] = s[live] + c * binv[xs]
        x[live] = b
        live = x != root
    return s


def fixed_point(values: np.ndarray) -> np.ndarray:
    return np.floor(values * float(1 << FRAC_BITS) + 0.5).astype(np.int64)


def accumulate(g, root: int, parents: np.ndarray) -> np.ndarray:
    """Signed fixed-point totals of S_T(v) over the trees (rows of parents)."""
    bpar, _ = bfs_tree(g, root)
    binv = bfs_inverse_weights(g, bpar)
    acc = np.zeros(g.n, dtype=np.int64)
    for par in np.atleast_2d(parents):
        acc += fixed_point(path_sums(g, root, bpar, binv, par))
    return acc


def resistance_from_totals(acc: np.ndarray, trees: int) -> np.ndarray:
    return acc.astype(np.float64) / (float(1 << FRAC_BITS) * trees)


def weighted_degrees(g) -> np.ndarray:
    """d_w(v): the row's weights (FP32 converted to FP64) summed left to right."""
    d = np.zeros(g.n)
    for v in range(g.n):
        s = 0.0
        for e in range(g.rowptr[v], g.rowptr[v + 1]):
            s = s + (1.0 if g.w is None else float(g.w[e]))
        d[v] = s
    return d


def resistance_from_visits(visits: np.ndarray, trees: int, dw: np.ndarray, root: int) -> np.ndarray:
    """The visit estimator (not in the paper): in Wilson's algorithm rooted at
    u the departures K_v from v in one tree do not depend on the start order,
    and taking v as the first start vertex shows that K_v is the number of
    visits to v of a walk from v killed at u, whose mean is the Green's
    function d_w(v) r(u, v).  So K_v / d_w(v) is unbiased for r(u, v):
    r^(u, v) = visits[v] / (trees d_w(v)), 0 at the root."""
    r = visits.astype(np.float64) / (float(trees) * dw)
    r[root] = 0.0
    return r


def pivot_column(g, root: int) -> np.ndarray:
    """x = L^+ e_root (insight (ii): one Laplacian solve; here the dense pinv)."""
    return laplacian_pinv(g)[:, root].copy()


def diag_from_resistance(r: np.ndarray, x: np.ndarray, root: int) -> np.ndarray:
    """Eq. 2 solved for L^+[v, v]: r(u, v) - x[u] + 2 x[v] with x = L^+ e_u."""
    return r - x[root] + 2.0 * x


def farness_from_diag(diag: np.ndarray) -> np.ndarray:
    """n L^+[v, v] + tr(L^+)."""
    return diag.size * diag + diag.sum()


# ---- brute force -------------------------------------------------------------
def spanning_trees_rooted(g, root: int):
    """Yield (parent array rooted at root, parent[root] = n; weight = product of
    the edge weights) for every spanning tree of G (tiny graphs only)."""
    n = g.n
    u, v, w = g.edges()
    w = np.ones(u.size) if w is None else w.astype(np.float64)
    E = [(int(a), int(b), float(c)) for a, b, c in zip(u, v, w)]
    for subset in itertools.combinations(range(len(E)), n - 1):
        uf = list(range(n))

        def find(a):
            while uf[a] != a:
                uf[a] = uf[uf[a]]
                a = uf[a]
            return a

        ok, weight = True, 1.0
        adj = [[] for _ in range(n)]
        for ei in subset:
            a, b, c = E[ei]
            ra, rb = find(a), find(b)
            if ra == rb:
                ok = False
                break
            uf[ra] = rb
            weight *= c
            adj[a].append(b)
            adj[b].append(a)
        if not ok:
            continue
        par = [-2] * n
        par[root] = n
        stack = [root]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if par[y] == -2:
                    par[y] = x
                    stack.append(y)
        yield np.array(par, dtype=np.int32), weight
