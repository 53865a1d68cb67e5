"""GPU electrical closeness on G (Sec. 3 insights (i)-(iii), Eq. 2, Def. 2 with
r) through the C ABI, against the CPU oracle.

Bars: bit-exact trees, step counts and BFS trees (integer work, identical
random stacks); bit-exact signed fixed-point path-sum totals (identical trees,
FP64 additions in the same order); 1e-9 relative for FP64 values computed from
identical totals and columns; the Laplacian solve against the dense
pseudo-inverse at its tolerance; the estimate against the dense L^+ within a
sampling bound."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import electrical as el
from oracle import native

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _connected(g):
    assert el.is_connected(g)
    return g


def _graphs():
    return {
        "ba": _connected(synth.barabasi_albert(3000, 3, 5)),
        "ba_w": _connected(synth.barabasi_albert(2500, 2, 6, weighted=True)),
        "er_w": _connected(synth.erdos_renyi(800, 10, 7, weighted=True)),
        "torus": synth.torus(40, 30),
        "path": synth.path(300),
        "star": synth.star(200),
        "k8": synth.complete(8),
    }


@pytest.mark.parametrize("name", ["ba", "ba_w", "er_w", "torus", "path", "star", "k8"])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_rooted_trees_bit_exact(name, kernel):
    """Uniform spanning trees of G rooted at a hub and at a low-degree vertex:
    parents and step counts equal the oracle's rooted sampler (the GPU counts
    the root's one step to u*), for the automatic, CSR-walk and edge-record
    kernels."""
    g = _graphs()[name]
    d = g.degrees()
    for root in (int(np.argmax(d)), int(np.argmin(d))):
        G = fc.Graph.rooted(g, root)
        G.set_kernel(kernel)
        tau = 24
        out = G.sample(77, tau, want_parents=True, want_steps=True)
        ref = native.wilson_rooted(g, root, seed=77, tau=tau)
        par = out["parents"][0].cpu().numpy()
        np.testing.assert_array_equal(par, ref["parents"])
        np.testing.assert_array_equal(out["steps"][0].cpu().numpy().astype(np.uint64), ref["steps"] + 1)
        R = out["R"].cpu().numpy()
        assert R[root] == tau and R.sum() == tau
        G.close()


def test_rooted_trees_bit_exact_in_clusters_and_bitmap_modes():
    g = _graphs()["ba_w"]
    root = int(np.argmax(g.degrees()))
    ref = native.wilson_rooted(g, root, seed=5, tau=8)
    for bitmap, cluster in ((1, 0), (2, 1), (3, 1), (2, 4), (0, 2)):
        G = fc.Graph.rooted(g, root)
        G.set_kernel(2)
        G.set_bitmap(bitmap)
        G.set_cluster(cluster)
        out = G.sample(5, 8, want_parents=True)
        np.testing.assert_array_equal(out["parents"][0].cpu().numpy(), ref["parents"], err_msg=str((bitmap, cluster)))
        G.close()


@pytest.mark.parametrize("name", ["ba", "ba_w", "er_w", "torus", "path", "star"])
def test_bfs_tree_matches_oracle(name):
    g = _graphs()[name]
    for root in (0, int(np.argmax(g.degrees())), g.n - 1):
        G = fc.Graph.rooted(g, root)
        par, dep = G.bfs_tree()
        bpar, depth = el.bfs_tree(g, root)
        np.testing.assert_array_equal(par.cpu().numpy(), bpar)
        np.testing.assert_array_equal(dep.cpu().numpy(), depth)
        G.close()


def test_rejects_disconnected_graphs_and_bad_roots():
    g = synth.from_edges(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5]))
    with pytest.raises(fc.FcError) as e:
        fc.Graph.rooted(g, 0)
    assert e.value.status == fc.FC_EINVAL and b"connected" in fc.lib().fc_last_error_message()
    gc = synth.path(5)
    for root in (-1, 5):
        with pytest.raises(fc.FcError):
            fc.Graph.rooted(gc, root)
    with pytest.raises(fc.FcError):
        fc.Graph.rooted(synth.empty(1), 0)
    # the diag(Omega) graphs have no pivot: the electrical entry points refuse them
    Gs = fc.Graph.from_csr(gc, [1.0])
    with pytest.raises(fc.FcError):
        Gs.resistance_accumulate(torch.zeros((1, 5), dtype=torch.int32, device="cuda"))
    with pytest.raises(fc.FcError):
        Gs.laplacian_solve(torch.zeros(5, dtype=torch.float64, device="cuda"))
    Gs.close()


@pytest.mark.parametrize("name", ["ba", "ba_w", "er_w", "torus", "path", "star", "k8"])
def test_resistance_totals_bit_exact(name):
    """Signed fixed-point path-sum totals over 70 trees (three chunks of the
    cooperative kernel, the last ragged) equal the oracle's, on the oracle's
    own trees and on the GPU's."""
    g = _graphs()[name]
    root = int(np.argmax(g.degrees()))
    tau = 70
    ref = native.wilson_rooted(g, root, seed=41, tau=tau)["parents"]
    exp = el.accumulate(g, root, ref)
    G = fc.Graph.rooted(g, root)
    acc = G.resistance_accumulate(torch.from_numpy(ref).cuda())
    np.testing.assert_array_equal(acc.cpu().numpy(), exp)
    out = G.sample(41, tau, want_parents=True)
    acc2 = G.resistance_accumulate(out["parents"][0])
    np.testing.assert_array_equal(acc2.cpu().numpy(), exp)
    # accumulation over calls: totals add
    acc3 = torch.zeros_like(acc2)
    G.resistance_accumulate(out["parents"][0][:30], acc=acc3)
    G.resistance_accumulate(out["parents"][0][30:], acc=acc3)
    assert torch.equal(acc3, acc2)
    G.close()


def test_resistance_accumulate_rejects_non_trees():
    g = _graphs()["ba"]
    root = 7
    G = fc.Graph.rooted(g, root)
    par = torch.from_numpy(native.wilson_rooted(g, root, seed=2, tau=1)["parents"]).cuda()
    for bad in ("root_not_on_ustar", "second_root", "cycle", "range"):
        p = par.clone()
        if bad == "root_not_on_ustar":
            p[0, root] = int(g.colidx[g.rowptr[root]])
        elif bad == "second_root":
            p[0, (root + 1) % g.n] = g.n
        elif bad == "cycle":
            a = int(g.colidx[g.rowptr[3]])
            p[0, 3] = a
            p[0, a] = 3
        else:
            p[0, 11] = g.n + 5
        with pytest.raises(fc.FcError) as e:
            G.resistance_accumulate(p)
        assert e.value.status == fc.FC_EINVAL, bad
    G.close()


@pytest.mark.parametrize("name", ["ba_w", "er_w", "torus", "path"])
def test_laplacian_solve_vs_dense_pinv(name):
    g = _graphs()[name]
    Lp = el.laplacian_pinv(g)
    G = fc.Graph.rooted(g, 0)
    cols = [0, int(np.argmax(g.degrees())), g.n // 2]
    B = torch.zeros((len(cols), g.n), dtype=torch.float64, device="cuda")
    for j, c in enumerate(cols):
        B[j, c] = 1.0
    X, _ = G.laplacian_solve(B, rel_tol=1e-12)
    X = X.cpu().numpy()
    for j, c in enumerate(cols):
        np.testing.assert_allclose(X[j], Lp[:, c], rtol=0, atol=1e-8 * np.abs(Lp[:, c]).max())
        assert abs(X[j].sum()) < 1e-9 * g.n
    # many right-hand sides (interleaved layout) and a b that does not sum to zero
    m = 40
    rng = np.random.default_rng(3)
    Bm = rng.standard_normal((m, g.n))
    Xm, _ = G.laplacian_solve(torch.from_numpy(Bm).cuda(), rel_tol=1e-12)
    np.testing.assert_allclose(Xm.cpu().numpy(), Bm @ Lp.T, rtol=0, atol=1e-7 * np.abs(Bm @ Lp.T).max())
    G.close()


@pytest.mark.parametrize("name", ["ba_w", "er_w", "torus"])
def test_electrical_closeness_vs_oracle_and_dense(name):
    """Combination from the same totals and the oracle's pivot column: r^,
    diag(L^+) (Eq. 2), farness and closeness within 1e-9 of the oracle; with
    the GPU's own column within 1e-7; the estimate against the dense L^+
    within a sampling bound."""
    g = _graphs()[name]
    root = int(np.argmax(g.degrees()))
    tau = 400
    G = fc.Graph.rooted(g, root)
    out = G.sample(9, tau, want_parents=True)
    acc = G.resistance_accumulate(out["parents"][0])
    xo = el.pivot_column(g, root)
    r, d, far, clo = G.electrical_closeness(acc, tau, torch.from_numpy(xo).cuda())
    ref = native.wilson_rooted(g, root, seed=9, tau=tau)["parents"]
    acc_o = el.accumulate(g, root, ref)
    r_o = el.resistance_from_totals(acc_o, tau)
    d_o = el.diag_from_resistance(r_o, xo, root)
    np.testing.assert_allclose(r.cpu().numpy(), r_o, rtol=1e-12, atol=0)
    np.testing.assert_allclose(d.cpu().numpy(), d_o, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(far.cpu().numpy(), el.farness_from_diag(d_o), rtol=1e-9)
    np.testing.assert_allclose(clo.cpu().numpy(), el.electrical_closeness(el.farness_from_diag(d_o)), rtol=1e-9)
    # the library's own pivot column
    e = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    e[root] = 1.0
    x, _ = G.laplacian_solve(e, rel_tol=1e-12)
    _, d2, _, _ = G.electrical_closeness(acc, tau, x)
    np.testing.assert_allclose(d2.cpu().numpy(), d_o, rtol=0, atol=1e-7)
    # against the definition: per-vertex spread of S_T over the same trees
    Lp = el.laplacian_pinv(g)
    bpar, _ = el.bfs_tree(g, root)
    binv = el.bfs_inverse_weights(g, bpar)
    S = np.stack([el.path_sums_np(g, root, bpar, binv, p) for p in ref[:100]])
    sd = S.std(axis=0, ddof=1).max() / math.sqrt(tau)
    assert np.max(np.abs(d2.cpu().numpy() - np.diag(Lp))) < 6 * sd + 1e-9
    G.close()


@pytest.mark.parametrize("name", ["ba", "ba_w", "er_w", "torus", "path", "star"])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_rooted_visit_totals_bit_exact(name, kernel):
    """Departures from every vertex summed over the trees (fc_sample_usts_ex)
    equal the oracle's; the root departs once per tree (to u*)."""
    g = _graphs()[name]
    root = int(np.argmax(g.degrees()))
    G = fc.Graph.rooted(g, root)
    G.set_kernel(kernel)
    tau = 40
    out = G.sample(13, tau, want_visits=True, with_C=False, want_steps=True)
    ref = native.wilson_rooted(g, root, seed=13, tau=tau, want_parents=False, want_visits=True)
    vis = out["visits"].cpu().numpy().astype(np.uint64)
    exp = ref["visits"].copy()
    exp[root] = tau
    np.testing.assert_array_equal(vis, exp)
    assert int(vis.sum()) == int(out["steps"].sum().item())
    G.close()


@pytest.mark.parametrize("weighted,alphas,kernel", [(False, [1.0], 2), (True, [0.3, 5.0], 2), (False, [1.0], 1),
                                                    (True, [1.0], 1)])
def test_augmented_visit_totals_bit_exact(weighted, alphas, kernel):
    """On G* the same output: departures from each vertex, per alpha."""
    g = synth.barabasi_albert(3000, 3, 7, weighted=weighted)
    G = fc.Graph.from_csr(g, alphas)
    G.set_kernel(kernel)
    out = G.sample(21, 30, want_visits=True)
    vis = out["visits"].cpu().numpy().astype(np.uint64).reshape(len(alphas), g.n)
    for a, al in enumerate(alphas):
        ref = native.wilson(g, al, seed=21, tau=30, alpha_idx=a, want_C=False, want_visits=True)
        np.testing.assert_array_equal(vis[a], ref["visits"])
    G.close()


@pytest.mark.parametrize("name", ["ba_w", "er_w", "torus"])
def test_electrical_closeness_from_visits(name):
    """The visit estimator through fc_electrical_closeness: equal to the
    oracle's (same totals, the oracle's column) to 1e-12 / 1e-9, and within a
    sampling bound of the dense L^+."""
    g = _graphs()[name]
    root = int(np.argmax(g.degrees()))
    tau = 400
    G = fc.Graph.rooted(g, root)
    out = G.sample(9, tau, want_visits=True, with_C=False)
    xo = el.pivot_column(g, root)
    r, d, far, clo = G.electrical_closeness(None, tau, torch.from_numpy(xo).cuda(), visits=out["visits"])
    ref = native.wilson_rooted(g, root, seed=9, tau=tau, want_parents=False, want_visits=True)
    dw = el.weighted_degrees(g)
    r_o = el.resistance_from_visits(ref["visits"], tau, dw, root)
    d_o = el.diag_from_resistance(r_o, xo, root)
    np.testing.assert_allclose(r.cpu().numpy(), r_o, rtol=1e-12, atol=0)
    np.testing.assert_allclose(d.cpu().numpy(), d_o, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(far.cpu().numpy(), el.farness_from_diag(d_o), rtol=1e-9)
    np.testing.assert_allclose(clo.cpu().numpy(), el.electrical_closeness(el.farness_from_diag(d_o)), rtol=1e-9)
    # against the definition: per-vertex spread of K_v / d_w(v) over 200 single trees
    K = np.stack([native.wilson_rooted(g, root, seed=9, tau=1, tree_offset=t, want_parents=False,
                                       want_visits=True)["visits"] for t in range(200)]).astype(np.float64) / dw
    sd = K.std(axis=0, ddof=1).max() / math.sqrt(tau)
    Lp = el.laplacian_pinv(g)
    assert np.max(np.abs(d.cpu().numpy() - np.diag(Lp))) < 6 * sd + 1e-9
    # exactly one estimate must be given
    with pytest.raises(fc.FcError):
        G.electrical_closeness(None, tau, torch.from_numpy(xo).cuda())
    G.close()


def test_full_size_ba_hub_pivot_bit_exact():
    """BA n = 2^20, m = 8 (the complex-network benchmark graph) rooted at its
    largest hub: the BFS tree, 4 trees and their path-sum totals equal the
    oracle's."""
    g = synth.barabasi_albert(1 << 20, 8, 2)
    root = int(np.argmax(g.degrees()))
    G = fc.Graph.rooted(g, root)
    par, dep = G.bfs_tree()
    bpar, depth = el.bfs_tree(g, root)
    np.testing.assert_array_equal(par.cpu().numpy(), bpar)
    np.testing.assert_array_equal(dep.cpu().numpy(), depth)
    tau = 4
    out = G.sample(2020, tau, want_parents=True, want_steps=True, want_visits=True)
    ref = native.wilson_rooted(g, root, seed=2020, tau=tau, want_visits=True)
    np.testing.assert_array_equal(out["parents"][0].cpu().numpy(), ref["parents"])
    np.testing.assert_array_equal(out["steps"][0].cpu().numpy().astype(np.uint64), ref["steps"] + 1)
    exp = ref["visits"].copy()
    exp[root] = tau
    np.testing.assert_array_equal(out["visits"].cpu().numpy().astype(np.uint64), exp)
    acc = G.resistance_accumulate(out["parents"][0])
    binv = el.bfs_inverse_weights(g, bpar)
    exp = sum(el.fixed_point(el.path_sums_np(g, root, bpar, binv, p)) for p in ref["parents"])
    np.testing.assert_array_equal(acc.cpu().numpy(), exp)
    G.close()


def test_full_size_ba_hub_benchmark_shape_bit_exact():
    """The electrical benchmark's sampler launch at full size: BA n = 2^20,
    m = 8 rooted at its largest hub, the automatic rooted shape (128 walkers
    per tree, tree membership as state flags, one CTA per tree, reverse
    breadth-first start order, the walker ramp), 152 trees at once: parents,
    step counts and visit totals equal the oracle's."""
    import concurrent.futures as cf
    g = synth.barabasi_albert(1 << 20, 8, 2)
    root = int(np.argmax(g.degrees()))
    G = fc.Graph.rooted(g, root)
    G.set_cluster(1)
    tau = 152
    out = G.sample(4242, tau, want_parents=True, want_steps=True, want_visits=True, with_C=False)
    assert G.last_kernel() == 2 and G.last_cluster() == 1
    assert G.last_shape()["walkers_per_tree"] == 128
    cuts = np.linspace(0, tau, 17).astype(int)
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        parts = list(ex.map(lambda ab: native.wilson_rooted(g, root, seed=4242, tau=int(ab[1] - ab[0]),
                                                            tree_offset=int(ab[0]), want_visits=True),
                            [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]))
    par = out["parents"][0].cpu().numpy()
    np.testing.assert_array_equal(par, np.concatenate([p["parents"] for p in parts]))
    steps = np.concatenate([p["steps"] for p in parts])
    np.testing.assert_array_equal(out["steps"][0].cpu().numpy().astype(np.uint64), steps + 1)
    exp = np.sum([p["visits"] for p in parts], axis=0, dtype=np.uint64)
    exp[root] = tau
    np.testing.assert_array_equal(out["visits"].cpu().numpy().astype(np.uint64), exp)
    G.close()
