"""Seeded graph generators producing simple undirected CSR graphs.

Every generator is a pure function of its arguments and seed (numpy PCG64).
Output contract (the input contract of the method, Sec. 2: finite, simple,
undirected, non-negative weights):
  * rowptr int64[n+1], colidx int32[nnz], rows sorted ascending,
  * no self-loops, no duplicate edges, symmetric (u in N(v) <=> v in N(u)),
  * w float32[nnz] or None (unweighted); w[u->v] == w[v->u].

Workload shapes (synthetic stand-ins for the paper's KONECT / OSM graphs, which
are not available here):
  * ``erdos_renyi``      - G(n, p) with p = avg_deg / (n - 1).
  * ``barabasi_albert``  - linear preferential attachment, m edges per new vertex,
                           seed clique K_{m+1}; heavy-tailed degrees ("complex").
  * ``perturbed_grid``   - 4-neighbour grid, a fraction of edges deleted uniformly,
                           plus a number of random local diagonal shortcuts,
                           weights U[1, 10] ("road").
  * ``rmat``             - R-MAT(a, b, c, d), Graph500-style label permutation.
  * ``torus``            - W x H 4-neighbour torus (closed-form spectrum).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Graph:
    n: int
    rowptr: np.ndarray  # int64[n+1]
    colidx: np.ndarray  # int32[nnz]
    w: np.ndarray | None = None  # float32[nnz] or None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)

    def edges(self):
        """Undirected edge list (u < v) with weights (or None)."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))
        dst = self.colidx.astype(np.int64)
        keep = src < dst
        return src[keep], dst[keep], (None if self.w is None else self.w[keep])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def from_edges(n: int, u, v, w=None, name: str = "") -> Graph:
    """Build a simple symmetric CSR from an undirected edge list.

    Self-loops are dropped; duplicate undirected edges keep the first weight.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.size:
        if u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n:
            raise ValueError("edge endpoint out of range")
    keep = u != v
    u, v = u[keep], v[keep]
    if w is not None:
        w = np.asarray(w, dtype=np.float32)[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = lo * n + hi
    if w is None:
        # unweighted: the sorted distinct keys give the same CSR as the general
        # path below (the (src, dst) pairs are distinct, so any sort orders them
        # the same way), with two plain sorts instead of argsorts
        ukey = np.sort(key)
        if ukey.size:
            ukey = ukey[np.concatenate(([True], ukey[1:] != ukey[:-1]))]
        lo, hi = ukey // n, ukey % n
        both = np.concatenate([ukey, hi * n + lo])
        both.sort()
        src, dst = both // n, both % n
        counts = np.bincount(src, minlength=n) if src.size else np.zeros(n, np.int64)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        return Graph(n=n, rowptr=rowptr, colidx=dst.astype(np.int32), w=None, name=name)
    _, first = np.unique(key, return_index=True)
    lo, hi = lo[first], hi[first]
    if w is not None:
        w = w[first]
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    ww = None if w is None else np.concatenate([w, w])
    order = np.argsort(src * n + dst, kind="stable")
    src, dst = src[order], dst[order]
    if ww is not None:
        ww = np.ascontiguousarray(ww[order], dtype=np.float32)
    counts = np.bincount(src, minlength=n) if src.size else np.zeros(n, np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Graph(n=n, rowptr=rowptr, colidx=dst.astype(np.int32), w=ww, name=name)


def _uniform_weights(rng, size, lo=1.0, hi=10.0):
    return rng.uniform(lo, hi, size=size).astype(np.float32)


def erdos_renyi(n: int, avg_deg: float, seed: int, weighted: bool = False) -> Graph:
    rng = _rng(seed)
    p = avg_deg / max(n - 1, 1)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.size) < p
    u, v = iu[keep], ju[keep]
    w = _uniform_weights(rng, u.size) if weighted else None
    return from_edges(n, u, v, w, name=f"er_n{n}_d{avg_deg:g}_s{seed}")


def barabasi_albert(n: int, m: int, seed: int, weighted: bool = False) -> Graph:
    """Linear preferential attachment (Batagelj-Brandes endpoint list).

    Vertices 0..m form a seed clique K_{m+1}.  Each later vertex v adds m edge
    slots; slot j picks a uniformly random earlier entry of the endpoint list, so
    targets are chosen with probability proportional to degree.  Picks that hit v
    itself or repeat a target are dropped when the simple graph is formed, so the
    realised average degree is slightly below 2m.
    """
    if n <= m + 1:
        iu, ju = np.triu_indices(n, k=1)
        return from_edges(n, iu, ju, None, name=f"ba_n{n}_m{m}_s{seed}")
    rng = _rng(seed)
    iu, ju = np.triu_indices(m + 1, k=1)
    seed_list = np.empty(2 * iu.size, dtype=np.int64)
    seed_list[0::2] = iu
    seed_list[1::2] = ju
    e0 = seed_list.size
    n_new = (n - m - 1) * m
    owner = (m + 1) + np.arange(n_new, dtype=np.int64) // m  # new endpoint of slot j
    # slot j occupies endpoint-list positions e0 + 2j (owner) and e0 + 2j + 1 (target)
    hi_excl = e0 + 2 * np.arange(n_new, dtype=np.int64)
    r = (rng.random(n_new) * hi_excl).astype(np.int64)
    r = np.minimum(r, hi_excl - 1)
    val = np.full(n_new, -1, dtype=np.int64)
    in_seed = r < e0
    val[in_seed] = seed_list[r[in_seed]]
    q = r - e0
    even = (~in_seed) & (q % 2 == 0)
    val[even] = owner[q[even] // 2]
    ptr = np.where((~in_seed) & (q % 2 == 1), (q - 1) // 2, -1)
    unresolved = np.nonzero(val < 0)[0]
    while unresolved.size:
        p = ptr[unresolved]
        got = val[p]
        done = got >= 0
        val[unresolved[done]] = got[done]
        nd = unresolved[~done]
        ptr[nd] = ptr[ptr[nd]]
        unresolved = nd
    u = np.concatenate([iu, owner])
    v = np.concatenate([ju, val])
    w = _uniform_weights(rng, u.size) if weighted else None
    return from_edges(n, u, v, w, name=f"ba_n{n}_m{m}_s{seed}")


def perturbed_grid(width: int, height: int, seed: int, delete_frac: float = 0.10,
                   shortcut_frac: float = 0.01, weighted: bool = True) -> Graph:
    """4-neighbour grid; delete ``delete_frac`` of the edges uniformly at random,
    then add ``round(shortcut_frac * |E_grid|)`` distinct random diagonal edges
    (x, y) - (x + 1, y +/- 1); weights U[1, 10] as float32."""
    rng = _rng(seed)
    n = width * height
    ys, xs = np.divmod(np.arange(n, dtype=np.int64), width)
    hmask = xs < width - 1
    vmask = ys < height - 1
    hu = np.nonzero(hmask)[0]
    vu = np.nonzero(vmask)[0]
    u = np.concatenate([hu, vu])
    v = np.concatenate([hu + 1, vu + width])
    e_grid = u.size
    n_del = int(round(delete_frac * e_grid))
    keep = np.ones(e_grid, dtype=bool)
    if n_del:
        keep[rng.permutation(e_grid)[:n_del]] = False
    u, v = u[keep], v[keep]
    n_sc = int(round(shortcut_frac * e_grid))
    su = np.empty(0, np.int64)
    sv = np.empty(0, np.int64)
    if n_sc and width > 1 and height > 1:
        have = set()
        keys = []
        while len(keys) < n_sc:
            k = 2 * (n_sc - len(keys)) + 16
            x = rng.integers(0, width - 1, size=k)
            y = rng.integers(0, height, size=k)
            up = rng.integers(0, 2, size=k).astype(bool)
            y2 = np.where(up, y + 1, y - 1)
            ok = (y2 >= 0) & (y2 < height)
            a = (y * width + x)[ok]
            b = (y2 * width + x + 1)[ok]
            for aa, bb in zip(a.tolist(), b.tolist()):
                key = (min(aa, bb), max(aa, bb))
                if key not in have:
                    have.add(key)
                    keys.append(key)
                    if len(keys) == n_sc:
                        break
        arr = np.array(keys, dtype=np.int64)
        su, sv = arr[:, 0], arr[:, 1]
    u = np.concatenate([u, su])
    v = np.concatenate([v, sv])
    w = _uniform_weights(rng, u.size) if weighted else None
    return from_edges(n, u, v, w, name=f"grid_{width}x{height}_s{seed}")


def torus(width: int, height: int, weight: float | None = None) -> Graph:
    """W x H 4-neighbour torus (W, H >= 3), optionally with a constant weight."""
    if width < 3 or height < 3:
        raise ValueError("torus needs width, height >= 3")
    n = width * height
    ys, xs = np.divmod(np.arange(n, dtype=np.int64), width)
    right = ys * width + (xs + 1) % width
    down = ((ys + 1) % height) * width + xs
    u = np.concatenate([np.arange(n), np.arange(n)])
    v = np.concatenate([right, down])
    w = None if weight is None else np.full(u.size, weight, dtype=np.float32)
    return from_edges(n, u, v, w, name=f"torus_{width}x{height}")


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
         permute: bool = True, chunk: int = 1 << 22) -> Graph:
    """R-MAT graph: 2^scale vertices, edge_factor * 2^scale sampled edges,
    symmetrised, deduplicated, self-loops dropped; labels permuted (Graph500)."""
    rng = _rng(seed)
    n = 1 << scale
    total = edge_factor * n
    ab, abc = a + b, a + b + c
    us, vs = [], []
    done = 0
    while done < total:
        k = min(chunk, total - done)
        uu = np.zeros(k, dtype=np.int64)
        vv = np.zeros(k, dtype=np.int64)
        q = np.empty(k, dtype=np.uint8)
        for lvl in range(scale):
            # quadrant of this level: 0 (a), 1 (b: v bit), 2 (c: u bit), 3 (d: both)
            r = rng.random(k)
            np.greater_equal(r, a, out=q, casting="unsafe")
            q += r >= ab
            q += r >= abc
            uu |= (q >> 1).astype(np.int64) << lvl
            vv |= (q & 1).astype(np.int64) << lvl
        us.append(uu)
        vs.append(vv)
        done += k
    u = np.concatenate(us)
    v = np.concatenate(vs)
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        u, v = perm[u], perm[v]
    return from_edges(n, u, v, None, name=f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def complete(n: int, weight: float | None = None) -> Graph:
    iu, ju = np.triu_indices(n, k=1)
    w = None if weight is None else np.full(iu.size, weight, np.float32)
    return from_edges(n, iu, ju, w, name=f"K{n}")


def path(n: int) -> Graph:
    return from_edges(n, np.arange(n - 1), np.arange(1, n), None, name=f"P{n}")


def cycle(n: int, weight: float | None = None) -> Graph:
    u = np.arange(n)
    v = (u + 1) % n
    w = None if weight is None else np.full(n, weight, np.float32)
    return from_edges(n, u, v, w, name=f"C{n}")


def star(n: int) -> Graph:
    return from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), None, name=f"S{n}")


def empty(n: int) -> Graph:
    return from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64), None, name=f"E{n}")


def random_small(n: int, p: float, seed: int, weighted: bool) -> Graph:
    """Small G(n, p) used by exhaustive tests."""
    rng = _rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.size) < p
    u, v = iu[keep], ju[keep]
    w = None
    if weighted:
        w = (rng.integers(1, 8, size=u.size) / 2.0).astype(np.float32)
    return from_edges(n, u, v, w, name=f"small_n{n}_s{seed}")


def uneven_batch(count: int, seed: int, n_min: int = 100, n_max: int = 50_000,
                 alpha_min: float = 0.1, alpha_max: float = 10.0):
    """A batch of ``count`` graphs: sizes log-uniform in [n_min, n_max]; half BA
    with m in {2..8}, half perturbed grids (closest square side, 10% deletions,
    1% shortcuts, unit weights dropped: unweighted); alpha log-uniform.

    Returns (graphs, alphas)."""
    rng = _rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count))
    alphas = np.exp(rng.uniform(math.log(alpha_min), math.log(alpha_max), size=count))
    graphs = []
    for i in range(count):
        nn = int(round(sizes[i]))
        gseed = int(rng.integers(0, 2**31))
        if i % 2 == 0:
            m = int(rng.integers(2, 9))
            graphs.append(barabasi_albert(nn, m, gseed))
        else:
            side = max(2, int(round(math.sqrt(nn))))
            graphs.append(perturbed_grid(side, side, gseed, weighted=False))
    return graphs, alphas


def union(graphs):
    """Block-diagonal union of graphs (vertex ids shifted); returns
    (Graph, vertex offsets int64[len(graphs)+1])."""
    offs = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        offs[i + 1] = offs[i] + g.n
    weighted = any(g.w is not None for g in graphs)
    rowptr = np.zeros(int(offs[-1]) + 1, dtype=np.int64)
    cols, ws = [], []
    e0 = 0
    for i, g in enumerate(graphs):
        rowptr[offs[i] + 1: offs[i + 1] + 1] = g.rowptr[1:] + e0
        cols.append(g.colidx.astype(np.int64) + offs[i])
        if weighted:
            ws.append(np.ones(g.nnz, np.float32) if g.w is None else g.w)
        e0 += g.nnz
    colidx = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    w = np.concatenate(ws).astype(np.float32) if weighted else None
    return Graph(n=int(offs[-1]), rowptr=rowptr, colidx=colidx, w=w, name=f"union{len(graphs)}"), offs
