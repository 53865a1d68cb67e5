"""Tree-path aggregation: forest roots/depths by BFS levels, and off-diagonal
Omega from root frequencies (matrix-forest theorem)."""
import numpy as np
import pytest
import scipy.stats
import torch

import synth
from oracle import dense, forest

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


@pytest.mark.parametrize("kind", ["er", "ba", "grid"])
def test_roots_and_depths_match_parent_walks(kind):
    if kind == "er":
        g, al = synth.erdos_renyi(1000, 8, 1), [1.0]
    elif kind == "ba":
        g, al = synth.barabasi_albert(20000, 4, 2), [0.5]
    else:
        g, al = synth.perturbed_grid(60, 50, 3), [10.0]
    G = fc.Graph.from_csr(g, al)
    out = G.sample(9, 6, want_parents=True)
    par = out["parents"][0]
    roots, depth = fc.tree_roots(par)
    r, d = roots.cpu().numpy(), depth.cpu().numpy()
    p = par.cpu().numpy()
    for t in range(p.shape[0]):
        rr, dd = forest.roots_and_depths_np(p[t])
        np.testing.assert_array_equal(r[t], rr)
        np.testing.assert_array_equal(d[t], dd)
    G.close()


def test_root_frequencies_estimate_omega_columns():
    g = synth.barabasi_albert(150, 2, 7, weighted=True)
    alpha = 0.8
    G = fc.Graph.from_csr(g, [alpha])
    tau = 20000
    out = G.sample(3, tau, want_parents=True)
    roots, _ = fc.tree_roots(out["parents"][0], want_depth=False)
    q = torch.tensor([0, 5, 77, 149], dtype=torch.int32, device="cuda")
    cnt = fc.root_counts(roots, q).cpu().numpy().view(np.uint32)
    R = out["R"].cpu().numpy().view(np.uint32)
    qn = q.cpu().numpy()
    np.testing.assert_array_equal(cnt[np.arange(qn.size), qn], R[qn])  # diagonal = u*-edge counts
    Om = dense.forest_matrix(g, alpha)
    est = cnt / tau
    ref = Om[qn, :]
    z = (est - ref) / np.sqrt(np.maximum(ref * (1 - ref), 1e-12) / tau)
    assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * z.size))
    # pairwise forest distance (Def. 1) from the same trees
    rho = est[1, qn[1]] + est[2, qn[2]] - 2 * est[1, qn[2]]
    assert abs(rho - dense.forest_distance(Om)[qn[1], qn[2]]) < 0.05
    G.close()


def test_tree_roots_rejects_non_trees():
    n = 6
    par = torch.tensor([[6, 0, 3, 2, 6, 4]], dtype=torch.int32, device="cuda")  # 2 <-> 3 cycle
    with pytest.raises(fc.FcError):
        fc.tree_roots(par)


def _check_forest(out, n_rows_graph, n):
    par = out["parents"].reshape(-1, n).cpu().numpy()
    roots = out["roots"].reshape(-1, n).cpu().numpy()
    depths = out["depths"].reshape(-1, n).cpu().numpy()
    for t in range(par.shape[0]):
        r, d = forest.roots_and_depths_np(par[t])
        np.testing.assert_array_equal(roots[t], r, err_msg=f"roots, tree row {t}")
        np.testing.assert_array_equal(depths[t], d, err_msg=f"depths, tree row {t}")


@pytest.mark.parametrize("case", ["ba_bitmap_prefix", "ba_flags_ring", "grid_flags_ring_weighted",
                                  "grid_bitmap_prefix_weighted", "ba_global_bitmap", "er_csr_walk",
                                  "ba_cluster_fallback", "rooted_ba"])
def test_fused_forest_roots_match_oracle(case):
    """Roots and depths written by the sampler as vertices join the tree (or by
    pointer jumping where the launch uses clusters or the CSR-walk kernel)
    equal the oracle's parent walks over the same trees, for every tree."""
    if case.startswith("grid"):
        g, al = synth.perturbed_grid(120, 100, 3), [0.3, 4.0]
    elif case.startswith("er"):
        g, al = synth.erdos_renyi(1500, 6, 4), [1.0]
    else:
        g, al = synth.barabasi_albert(30000, 5, 3), [1.0]
    if case == "rooted_ba":
        G = fc.Graph.rooted(g, int(np.argmax(g.degrees())))
    else:
        G = fc.Graph.from_csr(g, al)
    tau = 40
    if case != "er_csr_walk" and case != "rooted_ba":
        G.set_kernel(2)
        G.set_cluster(2 if case == "ba_cluster_fallback" else 1)
        G.set_bitmap({"bitmap": 2, "flags": 1, "global": 3, "cluster": 2}[case.split("_")[1]])
        G.set_pops(2 if "ring" in case else 1)
        G.set_shape(256, 0, 0, 64)
    elif case == "er_csr_walk":
        G.set_kernel(1)
    else:
        G.set_cluster(1)  # rooted: the fused path (40 trees would otherwise take clusters)
    out = G.sample(21, tau, want_parents=True, want_roots=True, with_C=False)
    expect_kernel = {"er_csr_walk": 1}.get(case)
    if expect_kernel:
        assert G.last_kernel() == expect_kernel
    if case == "ba_cluster_fallback":
        assert G.last_cluster() == 2
    _check_forest(out, tau, g.n)
    if case == "rooted_ba":
        root = int(np.argmax(g.degrees()))
        assert np.all(out["roots"].cpu().numpy() == root)
    # roots alone (depths from scratch) give the same roots
    out2 = G.sample(21, tau, want_roots=True, with_C=False)
    assert torch.equal(out2["roots"], out["roots"]) and torch.equal(out2["depths"], out["depths"])
    G.close()


def test_fused_forest_roots_batch():
    graphs, alphas = synth.uneven_batch(10, 5, n_min=40, n_max=500)
    u, offs = synth.union(graphs)
    G = fc.Graph.batch(u, offs, alphas)
    out = G.sample(4, 16, want_parents=True, want_roots=True, with_C=False)
    _check_forest(out, 16, u.n)
    G.close()


def test_fused_forest_roots_full_size_benchmark_shape():
    """BA n = 2^20, m = 8: the benchmark's launch shape (shipped table: 1024
    walkers, 64 registers, id order, in-tree bitmap in shared memory, one CTA
    per tree) with the forest written by the sampler; 40 trees against the
    oracle's parent walks."""
    g = synth.barabasi_albert(1 << 20, 8, 2)
    G = fc.Graph.from_csr(g, [1.0])
    G.set_shape(1024, 0, 0, 64)
    G.set_start_order("id")
    G.set_cluster(1)
    out = G.sample(77, 40, want_parents=True, want_roots=True, with_C=False)
    assert G.last_kernel() == 3 and G.last_cluster() == 1
    _check_forest(out, 40, g.n)
    G.close()
