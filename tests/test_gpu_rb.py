"""GPU Rao-Blackwellised estimator (fc_rb_accumulate) against the oracle: the
fixed-point sums are bit-exact on the same sampled trees (unweighted,
weighted, per-vertex alpha of a batch), the diag and farness follow, invalid
parent arrays are rejected, and at the benchmark size the estimate is far
tighter than the frequency of Prop. 1 on the same trees."""
import numpy as np
import pytest
import torch

import synth
from oracle import dense, native, rb

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _hubs(weighted):
    """ER plus two hubs joined to 700 and 300 vertices: rows longer than one
    256-entry segment."""
    base = synth.erdos_renyi(1000, 4, 13)
    u, v, _ = base.edges()
    rng = np.random.default_rng(14)
    hu = np.concatenate([np.zeros(700, np.int64), np.ones(300, np.int64)])
    hv = np.concatenate([rng.choice(np.arange(2, 1000), 700, replace=False),
                         rng.choice(np.arange(2, 1000), 300, replace=False)])
    u, v = np.concatenate([u, hu]), np.concatenate([v, hv])
    w = rng.uniform(0.25, 4.0, u.size).astype(np.float32) if weighted else None
    return synth.from_edges(1000, u, v, w)


@pytest.mark.parametrize("kind", ["er", "er_w", "grid_w", "ba_hubs_w", "isolated", "hubs", "hubs_w"])
def test_fixed_point_sums_bit_exact(kind):
    if kind == "er":
        g, alpha, tau = synth.erdos_renyi(1500, 6, 3), 1.0, 12
    elif kind == "er_w":
        g, alpha, tau = synth.erdos_renyi(1200, 5, 4, weighted=True), 0.6, 10
    elif kind == "grid_w":
        g, alpha, tau = synth.perturbed_grid(40, 35, 2), 3.0, 8
    elif kind == "ba_hubs_w":
        g, alpha, tau = synth.barabasi_albert(3000, 4, 5, weighted=True), 0.3, 6
    elif kind == "hubs":  # long unweighted rows split, three chunks of trees
        g, alpha, tau = _hubs(False), 0.7, 70
    elif kind == "hubs_w":  # long weighted rows, two chunks
        g, alpha, tau = _hubs(True), 0.4, 40
    else:
        base = synth.barabasi_albert(300, 2, 9)
        u, v, _ = base.edges()
        g, alpha, tau = synth.from_edges(700, u, v), 2.0, 10
    G = fc.Graph.from_csr(g, [alpha])
    out = G.sample(77, tau, want_parents=True)
    par = out["parents"][0]
    acc = G.rb_accumulate(par)
    ref = rb.accumulate(g, alpha, par.cpu().numpy())
    np.testing.assert_array_equal(_u64(acc), ref)
    d = G.rb_diag(acc, tau).cpu().numpy()
    np.testing.assert_array_equal(d, rb.diag_from_fixed(ref, tau))
    far, clo = G.farness_from_diag(torch.from_numpy(d).cuda())
    np.testing.assert_allclose(far.cpu().numpy(), dense.farness_eq3(d), rtol=1e-12)
    np.testing.assert_allclose(clo.cpu().numpy(), dense.closeness(dense.farness_eq3(d)), rtol=1e-12)
    # accumulating in two calls gives the same sums (order of trees does not matter)
    acc2 = G.rb_accumulate(par[tau // 2:])
    G.rb_accumulate(par[: tau // 2], acc=acc2)
    assert torch.equal(acc, acc2)
    G.close()


def test_batch_uses_each_graphs_alpha():
    graphs = [synth.barabasi_albert(400, 3, 1), synth.perturbed_grid(15, 12, 2), synth.erdos_renyi(200, 4, 3)]
    alphas = np.array([0.5, 4.0, 1.5])
    u, offs = synth.union(graphs)
    G = fc.Graph.batch(u, offs, alphas)
    tau = 16
    out = G.sample(5, tau, want_parents=True)
    par = out["parents"][0]
    acc = G.rb_accumulate(par)
    av = np.repeat(alphas, np.diff(offs))
    np.testing.assert_array_equal(_u64(acc), rb.accumulate(u, av, par.cpu().numpy()))
    G.close()


def test_invalid_parent_arrays_rejected():
    g = synth.erdos_renyi(300, 4, 1)
    G = fc.Graph.from_csr(g, [1.0])
    out = G.sample(3, 2, want_parents=True)
    par = out["parents"][0].clone()
    bad = par.clone()
    bad[0, 5] = g.n + 3  # out of range
    with pytest.raises(fc.FcError):
        G.rb_accumulate(bad)
    cyc = par.clone()
    cyc[1, 10], cyc[1, 11] = 11, 10  # a 2-cycle: not a tree rooted at u*
    with pytest.raises(fc.FcError):
        G.rb_accumulate(cyc)
    acc = G.rb_accumulate(par)  # the context is still usable
    np.testing.assert_array_equal(_u64(acc), rb.accumulate(g, 1.0, par.cpu().numpy()))
    G.close()


def test_benchmark_size_far_tighter_than_frequency():
    """BA n = 2^20, m = 8: 32 trees; both estimates against CG columns on
    degree-stratified vertices."""
    g = synth.barabasi_albert(1 << 20, 8, 2)
    G = fc.Graph.from_csr(g, [1.0])
    tau = 32
    out = G.sample(2024, tau, want_parents=True)
    d_rb = G.rb_diag(G.rb_accumulate(out["parents"][0]), tau)
    d_plain, _, _ = G.farness(out["R"], tau)
    rng = np.random.default_rng(1)
    deg = g.degrees()
    order = np.argsort(deg, kind="stable")
    J = np.unique(np.concatenate([order[:64], rng.choice(g.n, 192, replace=False)]))
    Jt = torch.from_numpy(J).cuda()
    B = torch.zeros(J.size, g.n, dtype=torch.float64, device="cuda")
    B[torch.arange(J.size, device="cuda"), Jt] = 1.0
    X, _ = G.solve(B, rel_tol=1e-10)
    om = X[torch.arange(J.size, device="cuda"), Jt]
    e_rb = (d_rb[Jt] - om).abs()
    e_pl = (d_plain[Jt] - om).abs()
    assert float(e_rb.max()) < 0.5 * float(e_pl.max())
    assert float((e_rb ** 2).mean()) < 0.05 * float((e_pl ** 2).mean())
    G.close()
