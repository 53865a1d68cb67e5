"""Pins of the electrical-closeness oracle (the diag(L^+) algorithm the paper
builds on, Sec. 3 insights (i)-(iii), Eq. 2, Def. 2 with r in place of the
forest distance) and of its rooted Wilson sampler.

Each function is checked against something other than itself: closed forms of
effective resistance, Foster's theorem, the defining identities of the
pseudo-inverse, scipy's shortest paths, brute-force enumeration of spanning
trees (exact expectation of the path sums; chi^2 of sampled tree
frequencies), and the Green's-function identity for the walk's visits."""
import math

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.csgraph
import scipy.stats

import synth
from oracle import dense, electrical as el, native


def _connected_small(n, p, seed, weighted):
    for s in range(seed, seed + 200):
        g = synth.random_small(n, p, s, weighted=weighted)
        if el.is_connected(g):
            return g
    raise RuntimeError("no connected sample")


def test_pinv_defining_identities():
    g = synth.barabasi_albert(60, 2, 4, weighted=True)
    L = dense.laplacian(g)
    Lp = el.laplacian_pinv(g)
    np.testing.assert_allclose(L @ Lp @ L, L, atol=1e-10)
    np.testing.assert_allclose(Lp @ L @ Lp, Lp, atol=1e-10)
    np.testing.assert_allclose(Lp, Lp.T, atol=1e-12)
    np.testing.assert_allclose(Lp.sum(axis=1), 0.0, atol=1e-10)
    np.testing.assert_allclose(Lp, np.linalg.pinv(L), atol=1e-9)


def test_resistance_closed_forms():
    # path with weights: r(0, k) = sum of 1 / w along the path
    n = 7
    w = np.array([1.0, 2.0, 0.5, 4.0, 3.0, 1.5], dtype=np.float32)
    g = synth.from_edges(n, np.arange(n - 1), np.arange(1, n), w)
    Lp = el.laplacian_pinv(g)
    for k in range(n):
        assert abs(el.resistance(Lp, 0, k) - float(np.sum(1.0 / w[:k].astype(np.float64)))) < 1e-12
    # cycle C_n (unit weights): r(0, k) = k (n - k) / n
    n = 11
    Lp = el.laplacian_pinv(synth.cycle(n))
    for k in range(n):
        assert abs(el.resistance(Lp, 0, k) - k * (n - k) / n) < 1e-12
    # complete graph K_n: r = 2 / n between distinct vertices
    Lp = el.laplacian_pinv(synth.complete(9))
    R = el.resistance_matrix(Lp)
    np.testing.assert_allclose(R[~np.eye(9, dtype=bool)], 2.0 / 9, atol=1e-12)
    np.testing.assert_allclose(np.diag(R), 0.0, atol=1e-12)
    # star: centre to leaf 1, leaf to leaf 2
    Lp = el.laplacian_pinv(synth.star(8))
    R = el.resistance_matrix(Lp)
    assert abs(R[0, 3] - 1.0) < 1e-12 and abs(R[2, 5] - 2.0) < 1e-12


def test_foster_theorem():
    """Sum over edges of w_e r(e) = n - 1 (Foster)."""
    for g in (synth.barabasi_albert(80, 3, 2, weighted=True), synth.perturbed_grid(9, 7, 1)):
        if not el.is_connected(g):
            continue
        R = el.resistance_matrix(el.laplacian_pinv(g))
        u, v, w = g.edges()
        w = np.ones(u.size) if w is None else w.astype(np.float64)
        assert abs(float(np.sum(w * R[u, v])) - (g.n - 1)) < 1e-9


def test_farness_identity_and_closeness():
    """Def. 2 with r: the sum of Eq. 2 over v equals n L^+[u,u] + tr(L^+);
    closeness = n / farness."""
    g = synth.barabasi_albert(50, 3, 9, weighted=True)
    Lp = el.laplacian_pinv(g)
    far = el.electrical_farness(Lp)
    brute = np.array([sum(el.resistance(Lp, u, v) for v in range(g.n) if v != u) for u in range(g.n)])
    np.testing.assert_allclose(far, brute, rtol=1e-12)
    np.testing.assert_allclose(el.farness_from_diag(np.diag(Lp)), brute, rtol=1e-11)
    np.testing.assert_allclose(el.electrical_closeness(far), g.n / brute, rtol=1e-12)
    # Eq. 2 solved for the diagonal from one column (insight (ii))
    for root in (0, 17):
        r = np.array([el.resistance(Lp, root, v) for v in range(g.n)])
        np.testing.assert_allclose(el.diag_from_resistance(r, Lp[:, root], root), np.diag(Lp), atol=1e-12)


def test_bfs_inverse_weights_by_edge_lookup():
    g = synth.barabasi_albert(200, 3, 8, weighted=True)
    bpar, _ = el.bfs_tree(g, 5)
    inv = el.bfs_inverse_weights(g, bpar)
    for v in range(g.n):
        exp = 0.0 if bpar[v] < 0 else 1.0 / float(np.float32(el.edge_weight(g, v, int(bpar[v]))))
        assert inv[v] == exp


def test_bfs_tree_against_scipy_shortest_paths():
    for g in (synth.barabasi_albert(300, 2, 7), synth.perturbed_grid(20, 15, 2)):
        A = scipy.sparse.csr_matrix((np.ones(g.nnz), g.colidx, g.rowptr), shape=(g.n, g.n))
        root = int(np.argmax(g.degrees()))
        hops = scipy.sparse.csgraph.shortest_path(A, unweighted=True, indices=root)
        bpar, depth = el.bfs_tree(g, root)
        reach = np.isfinite(hops)
        np.testing.assert_array_equal(depth[reach], hops[reach].astype(np.int64))
        assert np.all(depth[~reach] == -1)
        for v in np.nonzero(reach)[0]:
            if v == root:
                assert bpar[v] == -1
                continue
            nb = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
            closer = nb[hops[nb] == hops[v] - 1]
            assert bpar[v] == closer.min()


@pytest.mark.parametrize("n,p,seed,weighted", [(6, 0.6, 3, True), (6, 0.5, 11, False), (7, 0.45, 5, True),
                                               (5, 1.0, 2, False)])
def test_path_sums_exact_expectation_is_resistance(n, p, seed, weighted):
    """Kirchhoff: over ALL spanning trees of G weighted by the product of their
    edge weights, the expectation of S_T(v) is r(root, v) from the dense
    pseudo-inverse (Eq. 2), for every root and every vertex.  A dropped
    reverse-crossing term, a wrong sign or a wrong edge weight breaks it."""
    g = _connected_small(n, p, seed, weighted)
    Lp = el.laplacian_pinv(g)
    for root in range(g.n):
        bpar, _ = el.bfs_tree(g, root)
        binv = el.bfs_inverse_weights(g, bpar)
        num, tot = np.zeros(g.n), 0.0
        for par, wt in el.spanning_trees_rooted(g, root):
            num += wt * el.path_sums(g, root, bpar, binv, par)
            tot += wt
        r = np.array([el.resistance(Lp, root, v) for v in range(g.n)])
        np.testing.assert_allclose(num / tot, r, atol=1e-12)


def test_path_sums_on_a_tree_graph_are_deterministic():
    """A tree graph has one spanning tree: S_T(v) = r(root, v) exactly."""
    g = synth.barabasi_albert(40, 1, 3, weighted=True)
    root = 5
    o = native.wilson_rooted(g, root, seed=1, tau=1)
    s = el.path_sums(g, root, *(lambda b: (b, el.bfs_inverse_weights(g, b)))(el.bfs_tree(g, root)[0]),
                     o["parents"][0])
    Lp = el.laplacian_pinv(g)
    r = np.array([el.resistance(Lp, root, v) for v in range(g.n)])
    np.testing.assert_allclose(s, r, atol=1e-12)


def _key(par):
    return np.asarray(par, dtype=np.int32).tobytes()


@pytest.mark.parametrize("seed,weighted", [(3, False), (8, True), (21, True)])
def test_rooted_sampler_tree_frequencies(seed, weighted):
    """Wilson on G rooted at a vertex samples spanning trees with probability
    proportional to the product of the edge weights: chi^2 of 60k sampled
    parent arrays against brute-force enumeration."""
    g = _connected_small(5, 0.7, seed, weighted)
    root = 1
    trees = list(el.spanning_trees_rooted(g, root))
    total = sum(w for _, w in trees)
    dist = {_key(p): w / total for p, w in trees}
    tau = 60000
    out = native.wilson_rooted(g, root, seed=700 + seed, tau=tau)
    keys, counts = np.unique(out["parents"], axis=0, return_counts=True)
    got = {_key(k): c for k, c in zip(keys, counts)}
    assert set(got) <= set(dist)
    names = sorted(dist)
    obs = np.array([got.get(k, 0) for k in names], dtype=float)
    exp = np.array([dist[k] for k in names]) * tau
    small = exp < 5
    if small.any():
        obs = np.concatenate([obs[~small], [obs[small].sum()]])
        exp = np.concatenate([exp[~small], [exp[small].sum()]])
    assert scipy.stats.chisquare(obs, exp).pvalue > 1e-4


def test_rooted_sampler_order_invariance_and_spanning_trees():
    g = synth.barabasi_albert(300, 3, 5, weighted=True)
    root = 7
    a = native.wilson_rooted(g, root, seed=9, tau=6)
    b = native.wilson_rooted(g, root, seed=9, tau=6, order=np.random.default_rng(1).permutation(g.n))
    np.testing.assert_array_equal(a["parents"], b["parents"])
    np.testing.assert_array_equal(a["steps"], b["steps"])
    adj = [set(g.colidx[g.rowptr[v]:g.rowptr[v + 1]].tolist()) for v in range(g.n)]
    for par in a["parents"]:
        assert par[root] == g.n
        for v in range(g.n):
            if v != root:
                assert par[v] in adj[v]
            x, hops = v, 0
            while x != root:
                x = par[x]
                hops += 1
                assert hops <= g.n


def test_rooted_sampler_visits_match_greens_function():
    """Expected departures per tree = sum_v d_w(v) r(root, v) (visits to v of a
    walk killed at the root: d_w(v) r(root, v)), z-test over 4000 trees."""
    g = synth.barabasi_albert(60, 2, 13, weighted=True)
    root = 3
    tau = 4000
    o = native.wilson_rooted(g, root, seed=5, tau=tau)
    Lp = el.laplacian_pinv(g)
    dw = np.array([g.w[g.rowptr[v]:g.rowptr[v + 1]].astype(np.float64).sum() for v in range(g.n)])
    expect = float(np.sum(dw * np.array([el.resistance(Lp, root, v) for v in range(g.n)])))
    s = o["steps"].astype(np.float64)
    z = (s.mean() - expect) / (s.std(ddof=1) / math.sqrt(tau))
    assert abs(z) < 4.5, (s.mean(), expect)


def test_rooted_sampler_rejects_disconnected_graphs():
    g = synth.from_edges(5, np.array([0, 1, 3]), np.array([1, 2, 4]))
    with pytest.raises(ValueError):
        native.wilson_rooted(g, 0, seed=1, tau=1)


def test_sampled_estimator_unbiased_and_diag_within_bound():
    """r^ from sampled trees: per-vertex z-scores (Bonferroni) against Eq. 2;
    the diagonal from r^ and the exact pivot column within the matching bound;
    fixed-point totals equal the sum of the per-tree values."""
    g = synth.erdos_renyi(40, 5, 3, weighted=True)
    assert el.is_connected(g)
    root = int(np.argmax(g.degrees()))
    tau = 3000
    par = native.wilson_rooted(g, root, seed=17, tau=tau)["parents"]
    bpar, _ = el.bfs_tree(g, root)
    binv = el.bfs_inverse_weights(g, bpar)
    S = np.stack([el.path_sums(g, root, bpar, binv, p) for p in par])
    acc = el.accumulate(g, root, par)
    np.testing.assert_array_equal(acc, el.fixed_point(S).sum(axis=0))
    r_hat = el.resistance_from_totals(acc, tau)
    Lp = el.laplacian_pinv(g)
    r = np.array([el.resistance(Lp, root, v) for v in range(g.n)])
    sd = S.std(axis=0, ddof=1) / math.sqrt(tau)
    ok = sd > 0
    assert np.all(np.abs(r_hat - r)[~ok] < 1e-9)
    z = (r_hat - r)[ok] / sd[ok]
    assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * g.n))
    d_hat = el.diag_from_resistance(r_hat, el.pivot_column(g, root), root)
    assert np.max(np.abs(d_hat - np.diag(Lp))) < 6 * sd.max()


def test_vectorised_path_sums_equal_the_loop_bit_for_bit():
    """path_sums_np (numpy over all vertices at once) gives the same bits as
    the plain per-vertex loop, weighted and unweighted."""
    for g in (synth.barabasi_albert(400, 3, 4, weighted=True), synth.erdos_renyi(300, 6, 2),
              synth.perturbed_grid(15, 12, 4)):
        if not el.is_connected(g):
            continue
        for root in (0, int(np.argmax(g.degrees())), g.n - 1):
            bpar, _ = el.bfs_tree(g, root)
            binv = el.bfs_inverse_weights(g, bpar)
            for par in native.wilson_rooted(g, root, seed=3, tau=3)["parents"]:
                a = el.path_sums(g, root, bpar, binv, par)
                b = el.path_sums_np(g, root, bpar, binv, par)
                np.testing.assert_array_equal(a.view(np.uint64), b.view(np.uint64))


def test_visit_estimator_unbiased_per_vertex():
    """Departures from v in one rooted tree, divided by d_w(v), are unbiased for
    r(root, v) (Green's function of the walk killed at the root): per-vertex
    z-scores over 3000 trees (Bonferroni); the totals equal the step counts;
    the root departs never."""
    g = synth.barabasi_albert(60, 2, 21, weighted=True)
    root = 5
    T = 3000
    K = np.stack([native.wilson_rooted(g, root, seed=8, tau=1, tree_offset=t, want_parents=False,
                                       want_visits=True)["visits"] for t in range(T)]).astype(np.float64)
    tot = native.wilson_rooted(g, root, seed=8, tau=T, want_parents=False, want_visits=True)
    np.testing.assert_array_equal(tot["visits"], K.sum(axis=0).astype(np.uint64))
    assert int(tot["visits"].sum()) == int(tot["steps"].sum()) and tot["visits"][root] == 0
    dw = el.weighted_degrees(g)
    Lp = el.laplacian_pinv(g)
    r = np.array([el.resistance(Lp, root, v) for v in range(g.n)])
    X = K / dw
    r_hat = el.resistance_from_visits(tot["visits"], T, dw, root)
    np.testing.assert_allclose(r_hat, np.where(np.arange(g.n) == root, 0.0, X.mean(axis=0)), rtol=1e-12)
    m = np.arange(g.n) != root
    z = (r_hat - r)[m] / (X.std(axis=0, ddof=1)[m] / math.sqrt(T))
    assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * g.n))


def test_weighted_degrees_left_to_right():
    g = synth.barabasi_albert(100, 3, 2, weighted=True)
    dw = el.weighted_degrees(g)
    S = native.row_prefix(g)
    np.testing.assert_array_equal(dw, S[g.rowptr[1:] - 1])
