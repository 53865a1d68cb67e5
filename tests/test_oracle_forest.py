"""Pins of oracle/forest.py: the matrix-forest theorem over enumerated trees,
depths as tree distances (a library shortest-path routine), invariants and
special cases."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import synth
from oracle import dense, enumerate as oenum, forest, native


@pytest.mark.parametrize("name,alpha", [("K3", 1.0), ("path4w", 0.7), ("star5", 2.0), ("two_parts", 1.3)])
def test_root_shares_are_omega(name, alpha):
    # weighted share of spanning trees of G* in which root(v) = u equals
    # Omega[u, v] (the matrix-forest theorem, Sec. 2), Omega by a dense inverse
    if name == "K3":
        g = synth.complete(3)
    elif name == "path4w":
        g = synth.from_edges(4, [0, 1, 2], [1, 2, 3], [1.0, 2.5, 0.5])
    elif name == "star5":
        g = synth.star(5)
    else:
        g = synth.from_edges(5, [0, 2, 3], [1, 3, 4], [1.0, 3.0, 0.25])
    n = g.n
    num = np.zeros((n, n))
    total = 0.0
    for par, wt in oenum.spanning_trees(g, alpha):
        root, _ = forest.roots_and_depths(par)
        num[root, np.arange(n)] += wt
        total += wt
    omega = np.linalg.inv(np.eye(n) + alpha * dense.laplacian(g))
    np.testing.assert_allclose(num / total, omega, atol=1e-12)


def _tree_distances(par):
    n = par.size
    v = np.flatnonzero(par != n)
    A = sp.coo_matrix((np.ones(v.size), (v, par[v])), shape=(n, n)).tocsr()
    return csg.shortest_path(A, directed=False, unweighted=True)


def test_depths_are_tree_distances_and_invariants():
    g = synth.barabasi_albert(300, 3, 4)
    out = native.wilson(g, 0.8, seed=5, tau=6, want_parents=True)
    for par in out["parents"]:
        root, depth = forest.roots_and_depths(par)
        D = _tree_distances(par.astype(np.int64))
        np.testing.assert_array_equal(depth, D[np.arange(par.size), root].astype(np.int64))
        assert np.all(par[root] == g.n)                       # roots hang from u*
        np.testing.assert_array_equal(root[root], root)       # a root is its own root
        nr = par != g.n
        np.testing.assert_array_equal(root[par[nr]], root[nr])
        np.testing.assert_array_equal(depth[par[nr]], depth[nr] - 1)
        r2, d2 = forest.roots_and_depths_np(par)
        np.testing.assert_array_equal(r2, root)
        np.testing.assert_array_equal(d2, depth)


def test_special_cases():
    n = 7
    r, d = forest.roots_and_depths(np.full(n, n))        # every vertex a root
    np.testing.assert_array_equal(r, np.arange(n))
    np.testing.assert_array_equal(d, np.zeros(n))
    chain = np.array([1, 2, 3, 4, 5, 6, 7])                # 0 -> 1 -> ... -> 6 -> u*
    r, d = forest.roots_and_depths(chain)
    np.testing.assert_array_equal(r, np.full(n, 6))
    np.testing.assert_array_equal(d, 6 - np.arange(n))
    with pytest.raises(ValueError):
        forest.roots_and_depths(np.array([1, 0, 3]))       # 0 <-> 1 cycle
    with pytest.raises(ValueError):
        forest.roots_and_depths_np(np.array([1, 0, 3]))
