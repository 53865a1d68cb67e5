"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars: bit-exact for trees, counts and step counters (integer work, identical
random stacks); 1e-9 relative for FP64 per-vertex values computed from identical
counts; the paper's absolute eps for the estimate against dense inversion.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import cg as ocg
from oracle import cv as ocv
from oracle import dense, native

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _np32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _oracle_trees(g, alphas, seed, tau, tree_offset=0):
    outs = []
    for a, al in enumerate(alphas):
        outs.append(native.wilson(g, al, seed=seed, tau=tau, tree_offset=tree_offset, alpha_idx=a,
                                  want_parents=True))
    return outs


def _check_trees(G, g, alphas, seed, tau, tree_offset=0):
    out = G.sample(seed, tau, tree_offset=tree_offset, want_parents=True, want_steps=True)
    torch.cuda.synchronize()
    ref = _oracle_trees(g, alphas, seed, tau, tree_offset)
    n = g.n
    R = _np32(out["R"]).reshape(len(alphas), n)
    C = _np32(out["C"]).reshape(len(alphas), n)
    par = out["parents"].cpu().numpy()
    steps = out["steps"].cpu().numpy()
    for a in range(len(alphas)):
        np.testing.assert_array_equal(par[a], ref[a]["parents"], err_msg=f"parents alpha {a}")
        np.testing.assert_array_equal(R[a], ref[a]["R"], err_msg=f"R alpha {a}")
        np.testing.assert_array_equal(C[a], ref[a]["C"], err_msg=f"C alpha {a}")
        np.testing.assert_array_equal(steps[a].astype(np.uint64), ref[a]["steps"], err_msg=f"steps alpha {a}")
    return out, ref


@pytest.mark.parametrize("weighted,alphas", [(False, [1.0]), (False, [0.3, 4.0]), (True, [0.1, 1.0, 10.0])])
def test_stack_entries_bit_exact(weighted, alphas):
    g = synth.barabasi_albert(500, 4, 3, weighted=weighted)
    G = fc.Graph.from_csr(g, alphas)
    rng = np.random.default_rng(0)
    K = 20000
    verts = rng.integers(0, g.n, K).astype(np.int32)
    ks = rng.integers(0, 50, K).astype(np.uint32)
    for a, al in enumerate(alphas):
        for tree in (0, 7, 123456):
            got = G.stack_entries(99, tree, torch.from_numpy(verts).cuda(),
                                  torch.from_numpy(ks.view(np.int32)).cuda(), alpha_idx=a).cpu().numpy()
            ref = native.stack_entries(g, al, 99, tree, verts, ks, alpha_idx=a)
            np.testing.assert_array_equal(got, ref)
    G.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_p_root_bit_exact(weighted):
    g = synth.perturbed_grid(20, 15, 4, weighted=weighted)
    for alpha in (0.1, 1.0, 7.3):
        G = fc.Graph.from_csr(g, [alpha])
        got = G.p_root().cpu().numpy()
        np.testing.assert_array_equal(got, ocv.p_root(g, alpha))
        G.close()


@pytest.mark.parametrize("walkers,smem", [(0, 0), (32, 2), (64, 1), (256, 1), (1024, 2)])
def test_trees_bit_exact_er1000(walkers, smem):
    """Small configuration: ER G(1000, avg deg 8), alpha = 1, tau = 2000, every
    launch shape gives the oracle's trees."""
    g = synth.erdos_renyi(1000, 8, 1)
    G = fc.Graph.from_csr(g, [1.0])
    G.set_shape(walkers, 0, smem)
    tau = 2000 if walkers in (0, 64) else 300
    _check_trees(G, g, [1.0], seed=2021, tau=tau)
    G.close()


def test_trees_bit_exact_weighted_grid_three_alphas():
    g = synth.perturbed_grid(48, 40, 3)
    alphas = [0.1, 1.0, 10.0]
    G = fc.Graph.from_csr(g, alphas)
    for walkers, smem in ((0, 0), (128, 1)):
        G.set_shape(walkers, 0, smem)
        _check_trees(G, g, alphas, seed=7, tau=40)
    G.close()


@pytest.mark.parametrize("name", ["single", "empty", "star", "K8", "path", "two_parts", "isolated_mix"])
def test_trees_edge_cases(name):
    if name == "single":
        g = synth.empty(1)
    elif name == "empty":
        g = synth.empty(37)
    elif name == "star":
        g = synth.star(300)
    elif name == "K8":
        g = synth.complete(8, weight=2.5)
    elif name == "path":
        g = synth.path(500)
    elif name == "two_parts":
        g = synth.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5], [1.0, 2.0, 0.5, 3.0])
    else:
        base = synth.barabasi_albert(400, 2, 9)
        u, v, _ = base.edges()
        g = synth.from_edges(1000, u, v)  # vertices 400..999 isolated
    alphas = [0.5, 2.0]
    G = fc.Graph.from_csr(g, alphas)
    for walkers, smem in ((32, 2), (64, 1)):
        G.set_shape(walkers, 0, smem)
        out, ref = _check_trees(G, g, alphas, seed=11, tau=50)
    iso = g.degrees() == 0
    R = _np32(out["R"]).reshape(2, g.n)
    assert np.all(R[:, iso] == 50)
    G.close()


def test_tree_offset_split_equals_single_call():
    """Trees are indexed globally (resume / sharding identity)."""
    g = synth.barabasi_albert(3000, 3, 5)
    G = fc.Graph.from_csr(g, [1.0])
    full = G.sample(5, 96)
    R = torch.zeros_like(full["R"])
    C = torch.zeros_like(full["C"])
    G.sample(5, 40, tree_offset=0, R=R, C=C)
    G.sample(5, 56, tree_offset=40, R=R, C=C)
    assert torch.equal(R, full["R"]) and torch.equal(C, full["C"])
    G.close()


def test_ba_full_size_trees_bit_exact():
    """BA n = 2^20, m = 8, alpha = 1, few trees (the automatic shape spreads a
    tree over a thread-block cluster here): the first trees of the run are the
    oracle's, bit for bit."""
    g = synth.barabasi_albert(1 << 20, 8, 2)
    G = fc.Graph.from_csr(g, [1.0])
    _check_trees(G, g, [1.0], seed=12345, tau=3)
    # trees deep into the run (offset) as well
    _check_trees(G, g, [1.0], seed=12345, tau=1, tree_offset=1000)
    G.close()


def _oracle_threaded(g, alpha, seed, tau, tree_offset=0, alpha_idx=0, threads=16):
    """native.wilson over tree ranges in parallel host threads (the C sampler
    releases the GIL): parents, R, C and step counts of trees
    [tree_offset, tree_offset + tau), identical to one sequential call."""
    import concurrent.futures as cf
    threads = max(1, min(threads, tau))
    cuts = np.linspace(0, tau, threads + 1).astype(int)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(native.wilson, g, alpha, seed, int(b - a), tree_offset + int(a), alpha_idx, None, True)
                for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        parts = [f.result() for f in futs]
    return {"parents": np.concatenate([o["parents"] for o in parts]),
            "R": np.sum([o["R"] for o in parts], axis=0, dtype=np.uint32),
            "C": np.sum([o["C"] for o in parts], axis=0, dtype=np.uint32),
            "steps": np.concatenate([o["steps"] for o in parts])}


def _check_full_wave(G, g, alphas, seed, tau, tree_offset, expect_kernel, walkers, regs):
    out = G.sample(seed, tau, tree_offset=tree_offset, want_parents=True, want_steps=True)
    torch.cuda.synchronize()
    shape = G.last_shape()
    assert G.last_kernel() == expect_kernel and G.last_cluster() == 1, (G.last_kernel(), G.last_cluster())
    assert shape["walkers_per_tree"] == walkers and shape["regs"] == regs, shape
    # a full wave: one 1024-walker CTA per SM, every SM on its own tree at once
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert shape["ctas"] == min(nsm, len(alphas) * tau), (shape, nsm)
    n = g.n
    R = _np32(out["R"]).reshape(len(alphas), n)
    C = _np32(out["C"]).reshape(len(alphas), n)
    steps = out["steps"].cpu().numpy()
    for a, al in enumerate(alphas):
        ref = _oracle_threaded(g, al, seed, tau, tree_offset, a)
        par = out["parents"][a].cpu().numpy()
        for t in range(tau):
            np.testing.assert_array_equal(par[t], ref["parents"][t], err_msg=f"alpha {a} tree {t}")
        np.testing.assert_array_equal(R[a], ref["R"], err_msg=f"R alpha {a}")
        np.testing.assert_array_equal(C[a], ref["C"], err_msg=f"C alpha {a}")
        np.testing.assert_array_equal(steps[a].astype(np.uint64), ref["steps"], err_msg=f"steps alpha {a}")


def test_ba_full_size_benchmark_shape_full_wave_bit_exact():
    """The benchmark's own sampler launch: BA n = 2^20, m = 8 (seed 2), alpha = 1,
    the shipped tuning-table shape (1024 walkers per tree, 64-register variant,
    vertex-id start order), in-tree bitmap in shared memory, one CTA per tree,
    152 trees = one full wave of the persistent grid with every CTA on its own
    tree at once.  Parents, R, C and step counts of all 152 trees equal the
    oracle's, for the first wave of a step and for its last wave (trees
    872..1023 of a 1024-tree step)."""
    from paper_2101_06192_gb300 import tune
    g = synth.barabasi_albert(1 << 20, 8, 2)
    G = fc.Graph.from_csr(g, [1.0])
    entry = tune._load(tune._SHIPPED)[tune._key(G, 1024)]
    assert (entry["walkers"], entry["regs"], entry["order"]) == (1024, 64, "id")
    tune.apply(G, entry)
    G.set_cluster(1)
    for off in (0, 872):
        _check_full_wave(G, g, [1.0], seed=2024, tau=152, tree_offset=off, expect_kernel=3, walkers=1024, regs=64)
    G.close()


def test_grid_full_size_benchmark_shape_full_wave_bit_exact():
    """The road-like benchmark's sampler launch: 2048 x 2048 grid (10% deleted,
    1% diagonals, weights U[1, 10]), alpha in {0.1, 1, 10}; weighted edge-record
    kernel with tree membership as state flags, ring pops, degree start order,
    1024 walkers, 64 registers, one CTA per tree; 51 trees per alpha = 153 work
    items, more than one full wave of 152 CTAs.  Every tree equals the oracle's."""
    g = synth.perturbed_grid(2048, 2048, 3)
    alphas = [0.1, 1.0, 10.0]
    G = fc.Graph.from_csr(g, alphas)
    G.set_kernel(2)
    G.set_bitmap(1)
    G.set_pops(2)
    G.set_start_order("degree")
    G.set_shape(1024, 0, 0, 64)
    G.set_cluster(1)
    _check_full_wave(G, g, alphas, seed=33, tau=51, tree_offset=0, expect_kernel=2, walkers=1024, regs=64)
    G.close()


def test_grid_full_size_full_wave_repeatable():
    """Races show as trees that differ between runs of the same seed.  The
    2048 x 2048 weighted launch of the road-like benchmark (state flags, ring
    pops, 153 trees over 152 CTAs) three times: identical parents each time,
    and every parent is a grid neighbour (rows of 2048, diagonals included) or
    u*.  A missing warp barrier in the start-window compaction once lost a few
    start vertices per launch here (parent 0), depending on code generation."""
    g = synth.perturbed_grid(2048, 2048, 3)
    n = g.n
    vid = torch.arange(n, device="cuda", dtype=torch.int64)
    ok = torch.tensor([1, -1, 2048, -2048, 2047, -2047, 2049, -2049], device="cuda")
    first = None
    for _ in range(3):
        G = fc.Graph.from_csr(g, [0.1, 1.0, 10.0])
        G.set_kernel(2)
        G.set_bitmap(1)
        G.set_pops(2)
        G.set_start_order("degree")
        G.set_shape(1024, 0, 0, 64)
        G.set_cluster(1)
        par = G.sample(33, 51, want_parents=True)["parents"].reshape(-1, n).to(torch.int64)
        G.close()
        bad = (par != n) & ~torch.isin(par - vid, ok)
        assert int(bad.sum()) == 0, torch.nonzero(bad)[:4].tolist()
        if first is None:
            first = par
        else:
            assert torch.equal(par, first)
        del par


def test_grid_full_size_trees_bit_exact():
    """2048 x 2048 road-like grid, weights U[1, 10], alpha in {0.1, 1, 10}."""
    g = synth.perturbed_grid(2048, 2048, 3)
    alphas = [0.1, 1.0, 10.0]
    G = fc.Graph.from_csr(g, alphas)
    _check_trees(G, g, alphas, seed=3, tau=1)
    G.close()


def test_farness_and_closeness_vs_oracle_and_dense():
    g = synth.erdos_renyi(1000, 8, 1)
    tau = 2000
    G = fc.Graph.from_csr(g, [1.0])
    out = G.sample(2021, tau)
    diag, far, clo = G.farness(out["R"], tau)
    ref = native.wilson(g, 1.0, seed=2021, tau=tau)
    d_or = dense.diag_from_counts(ref["R"], tau)
    np.testing.assert_allclose(diag.cpu().numpy(), d_or, rtol=1e-12, atol=0)
    np.testing.assert_allclose(far.cpu().numpy(), dense.farness_eq3(d_or), rtol=1e-9)
    np.testing.assert_allclose(clo.cpu().numpy(), dense.closeness(dense.farness_eq3(d_or)), rtol=1e-9)
    # against the exact target (Thm. 1 with eps = 0.1)
    om = np.diag(dense.forest_matrix(g, 1.0))
    assert np.max(np.abs(diag.cpu().numpy() - om)) <= 0.1
    # the paper's fill step with the pivot solve reproduces R/tau
    x, _ = G.pivot_solve()
    diag2, _, _ = G.farness(out["R"], tau, x_pivot=x)
    np.testing.assert_allclose(diag2.cpu().numpy(), d_or, rtol=0, atol=1e-9)
    G.close()


def test_control_variate_combination_vs_oracle():
    g = synth.barabasi_albert(2000, 2, 8)
    tau = 500
    G = fc.Graph.from_csr(g, [1.0])
    out = G.sample(77, tau)
    gp = np.random.default_rng(1).random(g.n).astype(np.float32)
    diag, _, _ = G.farness(out["R"], tau, C=out["C"], g_pred=torch.from_numpy(gp).cuda())
    p = ocv.p_root(g, 1.0)
    ref = native.wilson(g, 1.0, seed=77, tau=tau)
    exp = ocv.combine(ref["R"], ref["C"], tau, p, ocv.beta_from_prediction(gp.astype(np.float64), p))
    np.testing.assert_allclose(diag.cpu().numpy(), exp, rtol=1e-9, atol=1e-12)
    G.close()


def test_control_variate_with_nonfinite_predictions():
    """Predictions that are NaN or infinite: NaN and -inf count as p_v, +inf as 1,
    exactly as the oracle's clip; the result stays finite everywhere."""
    g = synth.barabasi_albert(2000, 2, 9)
    tau = 300
    G = fc.Graph.from_csr(g, [1.0])
    out = G.sample(78, tau)
    gp = np.random.default_rng(2).random(g.n).astype(np.float32)
    gp[0::5] = np.nan
    gp[1::5] = np.inf
    gp[2::5] = -np.inf
    diag, far, _ = G.farness(out["R"], tau, C=out["C"], g_pred=torch.from_numpy(gp).cuda())
    p = ocv.p_root(g, 1.0)
    ref = native.wilson(g, 1.0, seed=78, tau=tau)
    exp = ocv.combine(ref["R"], ref["C"], tau, p, ocv.beta_from_prediction(gp.astype(np.float64), p))
    d = diag.cpu().numpy()
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(far.cpu().numpy()))
    np.testing.assert_allclose(d, exp, rtol=1e-9, atol=1e-12)
    G.close()


@pytest.mark.parametrize("weighted,alphas", [(False, [1.0]), (True, [0.3, 4.0])])
def test_visit_diag_vs_oracle_and_dense(weighted, alphas):
    """fc_visit_diag: visits / (tau deg*) equal to the oracle's to 1e-12 on
    the same (bit-exact) visit totals, and within a sampling bound of the dense
    diag(Omega); far below the indicator's error at the same tau."""
    g = synth.erdos_renyi(800, 8, 11, weighted=weighted)
    tau = 300
    G = fc.Graph.from_csr(g, alphas)
    out = G.sample(55, tau, want_visits=True)
    for a, al in enumerate(alphas):
        d = G.visit_diag(out["visits"], tau, alpha_idx=a).cpu().numpy()
        ref = native.wilson(g, al, seed=55, tau=tau, alpha_idx=a, want_C=False, want_visits=True)
        exp = dense.diag_from_visits(ref["visits"], tau, dense.deg_star(g, al))
        np.testing.assert_allclose(d, exp, rtol=1e-12, atol=0)
        om = np.diag(dense.forest_matrix(g, al))
        err_v = np.max(np.abs(d - om))
        err_r = np.max(np.abs(ref["R"] / tau - om))
        assert err_v < 0.5 * err_r, (err_v, err_r)
        assert err_v < 0.1
    G.close()


def test_visit_diag_batch_uses_each_graphs_alpha():
    graphs, alphas = synth.uneven_batch(12, 3, n_min=50, n_max=400)
    u, offs = synth.union(graphs)
    G = fc.Graph.batch(u, offs, alphas)
    tau = 64
    out = G.sample(8, tau, want_visits=True)
    d = G.visit_diag(out["visits"], tau).cpu().numpy()
    av = np.concatenate([np.full(gi.n, a) for gi, a in zip(graphs, alphas)])
    ref = native.wilson(u, av, seed=8, tau=tau, want_C=False, want_visits=True)
    np.testing.assert_array_equal(out["visits"].cpu().numpy().astype(np.uint64), ref["visits"])
    np.testing.assert_allclose(d, dense.diag_from_visits(ref["visits"], tau, dense.deg_star(u, av)), rtol=1e-12)
    G.close()


@pytest.mark.parametrize("kind,alpha", [("ba", 1.0), ("grid", 10.0), ("grid", 0.1)])
def test_solve_vs_oracle(kind, alpha):
    if kind == "ba":
        g = synth.barabasi_albert(3000, 4, 6, weighted=True)
    else:
        g = synth.perturbed_grid(50, 40, 2)
    G = fc.Graph.from_csr(g, [alpha])
    vs = np.array([0, 17, g.n // 2, g.n - 1])
    B = np.zeros((vs.size, g.n))
    B[np.arange(vs.size), vs] = 1.0
    X, iters = G.solve(torch.from_numpy(B).cuda(), rel_tol=1e-10)
    ref = ocg.omega_columns(g, alpha, vs).T
    np.testing.assert_allclose(X.cpu().numpy(), ref, atol=1e-9 * np.abs(ref).max())
    A = ocg.system_matrix(g, alpha)
    res = B.T - A @ X.cpu().numpy().T
    assert np.all(np.linalg.norm(res, axis=0) <= 1e-10 * np.linalg.norm(B.T, axis=0) * 1.01)
    G.close()


@pytest.mark.parametrize("kind,alpha", [("ba", 1.0), ("grid", 0.1)])
def test_solve_single_rhs_vs_oracle(kind, alpha):
    # one right-hand side: the inner CG runs as one cooperative launch that
    # sums its block partials in a fixed order, so repeated solves agree bit for bit
    g = synth.barabasi_albert(20000, 4, 7, weighted=True) if kind == "ba" else synth.perturbed_grid(150, 140, 3)
    G = fc.Graph.from_csr(g, [alpha])
    v = g.n // 3
    b = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    b[v] = 1.0
    x, iters = G.solve(b, rel_tol=1e-10)
    x2, iters2 = G.solve(b, rel_tol=1e-10)
    assert iters == iters2 and torch.equal(x, x2)
    ref = ocg.omega_columns(g, alpha, np.array([v]))[:, 0]
    np.testing.assert_allclose(x.cpu().numpy(), ref, atol=1e-9 * np.abs(ref).max())
    A = ocg.system_matrix(g, alpha)
    assert np.linalg.norm(b.cpu().numpy() - A @ x.cpu().numpy()) <= 1e-10 * 1.01
    # too few iterations: FC_ENOCONV
    with pytest.raises(fc.FcError) as e:
        G.solve(b, rel_tol=1e-14, max_iter=3)
    assert e.value.status == fc.FC_ENOCONV
    G.close()


def test_solve_single_rhs_hubs_and_empty_rows():
    # rows of 0 entries between others (the tiles' general walk), rows of
    # thousands of entries spread over many tiles, and a ragged last tile
    rng = np.random.default_rng(11)
    n = 9000
    hubs = np.array([5, 4000, 8999])
    u = [np.repeat(hubs, [3000, 700, 2600]), rng.integers(0, n, 6000)]
    v = [rng.choice(n, 3000, replace=False), rng.choice(n, 700, replace=False), rng.choice(n, 2600, replace=False),
         rng.integers(0, n, 6000)]
    u = np.concatenate(u)
    v = np.concatenate(v)
    keep = (u != v) & ~np.isin(u, np.arange(2000, 2600)) & ~np.isin(v, np.arange(2000, 2600))
    g = synth.from_edges(n, u[keep], v[keep], rng.uniform(0.5, 4.0, keep.sum()))
    assert (np.diff(g.rowptr) == 0).sum() >= 600 and g.nnz % 256 != 0
    G = fc.Graph.from_csr(g, [3.0])
    vs = [5, 2100, 8000]
    B = np.zeros((len(vs), n))
    B[np.arange(len(vs)), vs] = 1.0
    ref = ocg.omega_columns(g, 3.0, vs)
    for j in range(len(vs)):
        x, _ = G.solve(torch.from_numpy(B[j]).cuda(), rel_tol=1e-11)
        np.testing.assert_allclose(x.cpu().numpy(), ref[:, j], atol=1e-10 * np.abs(ref[:, j]).max())
    G.close()


def test_pivot_solve_closed_form():
    g = synth.barabasi_albert(5000, 3, 4, weighted=True)
    G = fc.Graph.from_csr(g, [2.0])
    x, _ = G.pivot_solve(rel_tol=1e-12)
    x = x.cpu().numpy()
    n = g.n
    np.testing.assert_allclose(x[:n] - x[n], -1.0 / (n + 1), atol=1e-12)
    assert abs(x.sum()) < 1e-9
    G.close()


def test_top_k_matches_oracle_with_ties():
    g = synth.erdos_renyi(1000, 8, 1)
    G = fc.Graph.from_csr(g, [1.0])
    tau = 64  # coarse counts: many exact ties
    out = G.sample(1, tau)
    diag, _, _ = G.farness(out["R"], tau)
    d = diag.cpu().numpy()
    for k in (1, 10, 500, 1000):
        np.testing.assert_array_equal(fc.top_k(diag, k).cpu().numpy(), dense.top_k(d, k))
    dd = torch.tensor([-1.0, 2.0, -3.5, -0.0, 0.0, 2.0, float("inf"), float("nan")], dtype=torch.float64,
                      device="cuda")
    assert fc.top_k(dd, 8).cpu().tolist() == [2, 0, 3, 4, 1, 5, 6, 7]
    np.testing.assert_array_equal(fc.top_k(dd, 8).cpu().numpy(), dense.top_k(dd.cpu().numpy(), 8))
    G.close()


@pytest.mark.parametrize("bad", ["unsorted", "self_loop", "asym", "neg_w", "nan_w", "col_range", "rowptr"])
def test_invalid_csr_rejected(bad):
    g = synth.random_small(8, 0.6, 1, weighted=True)
    rp, ci, w = g.rowptr.copy(), g.colidx.copy(), g.w.copy()
    if bad == "unsorted":
        v = int(np.argmax(np.diff(rp) >= 2))
        a = rp[v]
        ci[a], ci[a + 1] = ci[a + 1], ci[a]
    elif bad == "self_loop":
        ci[rp[2]] = 2
    elif bad == "asym":
        w[0] = w[0] + 1.0
    elif bad == "neg_w":
        w[3] = -1.0
    elif bad == "nan_w":
        w[3] = np.nan
    elif bad == "col_range":
        ci[-1] = 8
    else:
        rp[3] = rp[-1] + 10
    with pytest.raises(fc.FcError) as e:
        fc.Graph(rp, ci, w, [1.0])
    assert e.value.status == fc.FC_EINVAL
    # the device is still usable
    G = fc.Graph.from_csr(g, [1.0])
    G.sample(1, 4)
    G.close()


def test_bad_alpha_rejected():
    g = synth.path(5)
    for al in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(fc.FcError):
            fc.Graph.from_csr(g, [al])


def test_watchdog_returns_timeout_and_device_recovers():
    g = synth.barabasi_albert(20000, 4, 1)
    G = fc.Graph.from_csr(g, [1.0])
    G.set_shape(64, 0, 1)
    with pytest.raises(fc.FcError) as e:
        G.sample(3, 8, max_steps_per_tree=5)
    assert e.value.status == fc.FC_ETIMEOUT
    out = G.sample(3, 8, want_steps=True)
    ref = native.wilson(g, 1.0, seed=3, tau=8)
    np.testing.assert_array_equal(_np32(out["R"]), ref["R"])
    G.close()
