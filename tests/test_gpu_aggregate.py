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
