"""The edge-record sampler kernel (unweighted single graphs, one dependent
round trip per walk step) against the oracle: bit-exact trees, counts and step
counters for every start order and launch shape, including the edge cases of
the graph (isolated vertices, stars, paths) and of the walk (long paths that
overflow the remembered prefix, many colliding walkers)."""
import numpy as np
import pytest
import torch

import synth
from oracle import native

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _np32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _check(G, g, alphas, seed, tau, tree_offset=0):
    out = G.sample(seed, tau, tree_offset=tree_offset, want_parents=True, want_steps=True)
    torch.cuda.synchronize()
    assert G.last_kernel() in (2, 3, 4)
    n = g.n
    R = _np32(out["R"]).reshape(len(alphas), n)
    C = _np32(out["C"]).reshape(len(alphas), n)
    par = out["parents"].cpu().numpy()
    steps = out["steps"].cpu().numpy()
    for a, al in enumerate(alphas):
        ref = native.wilson(g, al, seed=seed, tau=tau, tree_offset=tree_offset, alpha_idx=a, want_parents=True)
        np.testing.assert_array_equal(par[a], ref["parents"], err_msg=f"parents alpha {a}")
        np.testing.assert_array_equal(R[a], ref["R"], err_msg=f"R alpha {a}")
        np.testing.assert_array_equal(C[a], ref["C"], err_msg=f"C alpha {a}")
        np.testing.assert_array_equal(steps[a].astype(np.uint64), ref["steps"], err_msg=f"steps alpha {a}")
    return out


@pytest.mark.parametrize("order", ["id", "id_desc", "degree", "degree_desc"])
@pytest.mark.parametrize("walkers,regs", [(0, 0), (32, 40), (256, 48), (1024, 64)])
@pytest.mark.parametrize("bitmap", [1, 2, 3])  # state flags, shared-memory bitmap, global bitmap
def test_er_trees_bit_exact(order, walkers, regs, bitmap):
    g = synth.erdos_renyi(1000, 8, 1)
    G = fc.Graph.from_csr(g, [1.0])
    G.set_kernel(2)
    G.set_shape(walkers, 0, 0, regs)
    G.set_bitmap(bitmap)
    G.set_start_order(order)
    _check(G, g, [1.0], seed=2021, tau=200)
    assert G.last_kernel() == bitmap + 1
    G.close()


@pytest.mark.parametrize("kind", ["ba", "grid_small_alpha", "torus", "rmat"])
def test_graph_families_bit_exact(kind):
    if kind == "ba":
        g, alphas, tau = synth.barabasi_albert(3000, 3, 5), [1.0], 64
    elif kind == "grid_small_alpha":
        # long walks (alpha small): paths longer than the remembered prefix
        g, alphas, tau = synth.perturbed_grid(60, 50, 4, weighted=False), [0.02, 3.0], 24
    elif kind == "torus":
        g, alphas, tau = synth.torus(40, 30), [0.05], 24
    else:
        g, alphas, tau = synth.rmat(12, 8, 3), [0.5, 8.0], 32
    G = fc.Graph.from_csr(g, alphas)
    G.set_kernel(2)
    for walkers, bitmap, pops in ((0, 1, 1), (512, 1, 2), (0, 2, 2), (1024, 2, 1), (256, 3, 1), (1024, 3, 2)):
        G.set_shape(walkers, 0, 0)
        G.set_bitmap(bitmap)
        G.set_pops(pops)
        _check(G, g, alphas, seed=99, tau=tau)
        assert G.last_kernel() == bitmap + 1
    G.close()


@pytest.mark.parametrize("name", ["single", "empty", "star", "path", "K8", "isolated_mix"])
def test_edge_cases_bit_exact(name):
    if name == "single":
        g = synth.empty(1)
    elif name == "empty":
        g = synth.empty(37)
    elif name == "star":
        g = synth.star(300)
    elif name == "path":
        g = synth.path(500)
    elif name == "K8":
        g = synth.complete(8)
    else:
        base = synth.barabasi_albert(400, 2, 9)
        u, v, _ = base.edges()
        g = synth.from_edges(1000, u, v)
    alphas = [0.5, 2.0]
    G = fc.Graph.from_csr(g, alphas)
    if g.nnz == 0:
        # no edge records without edges: the automatic choice is the CSR-walk kernel
        with pytest.raises(fc.FcError):
            G.set_kernel(2)
        G.close()
        return
    G.set_kernel(2)
    for walkers, smem, bitmap in ((32, 1, 0), (64, 1, 0), (32, 0, 0), (64, 0, 0), (64, 0, 3)):
        G.set_shape(walkers, 0, smem)
        G.set_bitmap(bitmap)
        out = _check(G, g, alphas, seed=11, tau=50)
    iso = g.degrees() == 0
    R = _np32(out["R"]).reshape(2, g.n)
    assert np.all(R[:, iso] == 50)
    G.close()


def test_both_kernels_agree_and_default_is_edge_kernel():
    g = synth.barabasi_albert(50_000, 4, 8)
    G = fc.Graph.from_csr(g, [1.0])
    outs = []
    for k in (0, 1, 2):
        G.set_kernel(k)
        o = G.sample(4, 64, want_parents=True, want_steps=True)
        torch.cuda.synchronize()
        outs.append((k, G.last_kernel(), o))
    assert outs[0][1] in (2, 3, 4) and outs[1][1] == 1 and outs[2][1] in (2, 3, 4)
    for key in ("parents", "R", "C", "steps"):
        for _, _, o in outs[1:]:
            assert torch.equal(o[key], outs[0][2][key]), key
    G.close()


@pytest.mark.parametrize("kind", ["grid", "grid_small_alpha", "K8", "ba_hubs", "two_parts"])
@pytest.mark.parametrize("bitmap", [1, 2, 3])
def test_weighted_trees_bit_exact(kind, bitmap):
    """Weighted graphs: slot thresholds carried in the 64-byte records; rows
    with more than 13 slots (BA hubs) search the rest of B in global memory."""
    if kind == "grid":
        g, alphas, tau = synth.perturbed_grid(48, 40, 3), [0.1, 1.0, 10.0], 24
    elif kind == "grid_small_alpha":
        g, alphas, tau = synth.perturbed_grid(40, 30, 5), [0.02, 30.0], 16
    elif kind == "K8":
        g, alphas, tau = synth.complete(8, weight=2.5), [0.5, 2.0], 64
    elif kind == "ba_hubs":
        g, alphas, tau = synth.barabasi_albert(4000, 4, 6, weighted=True), [0.3, 3.0], 32
        assert g.degrees().max() > 13
    else:
        g, alphas, tau = synth.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5], [1.0, 2.0, 0.5, 3.0]), [0.5, 2.0], 64
    G = fc.Graph.from_csr(g, alphas)
    G.set_kernel(2)
    G.set_bitmap(bitmap)
    for walkers, pops in ((32, 2), (256, 1), (256, 2)):
        G.set_shape(walkers, 0, 0)
        G.set_pops(pops)
        _check(G, g, alphas, seed=41, tau=tau)
        assert G.last_kernel() == bitmap + 1
    G.close()


@pytest.mark.parametrize("bitmap", [1, 2, 3])
def test_edge_kernel_watchdog_and_recovery(bitmap):
    g = synth.barabasi_albert(20000, 4, 1)
    G = fc.Graph.from_csr(g, [1.0])
    G.set_kernel(2)
    G.set_bitmap(bitmap)
    G.set_shape(64, 0, 0)
    with pytest.raises(fc.FcError) as e:
        G.sample(3, 8, max_steps_per_tree=5)
    assert e.value.status == fc.FC_ETIMEOUT
    out = G.sample(3, 8)
    ref = native.wilson(g, 1.0, seed=3, tau=8)
    np.testing.assert_array_equal(_np32(out["R"]), ref["R"])
    G.close()


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("bitmap", [1, 2])
def test_cluster_trees_bit_exact(cluster, bitmap):
    """Trees shared by the CTAs of a thread-block cluster (walkers, start
    windows and, with the shared-memory bitmap, the bitmap split over the
    CTAs' shared memories) give the oracle's trees."""
    cases = [(synth.barabasi_albert(20000, 4, 3), [1.0], 16),
             (synth.perturbed_grid(90, 70, 5), [0.2, 6.0], 8),
             (synth.erdos_renyi(3000, 5, 9), [0.7], 24)]
    for g, alphas, tau in cases:
        G = fc.Graph.from_csr(g, alphas)
        G.set_kernel(2)
        G.set_bitmap(bitmap)
        G.set_cluster(cluster)
        for walkers in (64, 256):
            G.set_shape(walkers, 0, 0)
            _check(G, g, alphas, seed=5, tau=tau)
            assert G.last_cluster() == cluster
            assert G.last_kernel() == bitmap + 1
        G.close()


def test_bitmap_split_over_cluster_for_large_graph():
    """2.1 M vertices: the in-tree bitmap (262 KB) fits in shared memory only
    when split over a cluster; the automatic cluster grows until it does."""
    g = synth.torus(1448, 1448)
    G = fc.Graph.from_csr(g, [0.5])
    G.set_kernel(2)
    G.set_bitmap(2)
    G.set_shape(256, 0, 0)
    _check(G, g, [0.5], seed=8, tau=2)
    assert G.last_cluster() >= 2 and G.last_kernel() == 3
    G.close()


def test_automatic_cluster_for_few_trees():
    g = synth.barabasi_albert(50_000, 4, 2)
    G = fc.Graph.from_csr(g, [1.0])
    _check(G, g, [1.0], seed=3, tau=4)   # 4 trees: clusters of 8 CTAs
    assert G.last_cluster() == 8
    _check(G, g, [1.0], seed=3, tau=300)  # enough trees: one CTA each
    assert G.last_cluster() == 1
    G.close()


def test_automatic_cluster_keeps_every_tree_in_flight():
    """16 trees: 16 x 8 CTAs fit the SM count, but clusters are placed within a
    GPC and fewer clusters of 8 are resident; the automatic cluster is halved
    until the whole launch runs in one wave.  Trees still equal the oracle's."""
    g = synth.barabasi_albert(50_000, 4, 2)
    G = fc.Graph.from_csr(g, [1.0])
    _check(G, g, [1.0], seed=5, tau=16)
    cl = G.last_cluster()
    assert cl in (4, 8), cl
    assert G.last_shape()["ctas"] == 16 * cl, (G.last_shape(), cl)
    G.close()
