"""Batches of graphs (fc_build_batch): one launch samples tau trees of every
graph.  The trees must equal the oracle's on the block-diagonal union with each
vertex carrying its graph's alpha, and farness/closeness are per graph."""
import numpy as np
import pytest
import torch

import synth
from oracle import dense, native

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _batch(seed=1):
    rng = np.random.default_rng(seed)
    graphs = [synth.barabasi_albert(300, 3, 1), synth.perturbed_grid(12, 10, 2), synth.erdos_renyi(150, 4, 3),
              synth.star(40), synth.empty(5), synth.barabasi_albert(800, 2, 4, weighted=True),
              synth.path(60), synth.complete(9, weight=2.0)]
    alphas = rng.uniform(0.2, 8.0, size=len(graphs))
    u, offs = synth.union(graphs)
    return graphs, alphas, u, offs


@pytest.mark.parametrize("walkers,smem,kernel,bitmap", [(0, 0, 0, 0), (64, 1, 1, 0), (32, 2, 1, 0),
                                                        (64, 0, 2, 2), (256, 0, 2, 1), (128, 0, 2, 3)])
def test_batch_trees_match_union_oracle(walkers, smem, kernel, bitmap):
    """Both sampler kernels: the CSR-walk kernel (state in shared or global
    memory) and the edge-record kernel with each tree-membership mode."""
    graphs, alphas, u, offs = _batch()
    G = fc.Graph.batch(u, offs, alphas)
    G.set_shape(walkers, 0, smem)
    if kernel:
        G.set_kernel(kernel)
    G.set_bitmap(bitmap)
    tau = 24
    out = G.sample(99, tau, want_parents=True, want_steps=True)
    av = np.repeat(alphas, np.diff(offs))
    ref = native.wilson(u, av, seed=99, tau=tau, want_parents=True)
    np.testing.assert_array_equal(out["parents"][0].cpu().numpy(), ref["parents"])
    np.testing.assert_array_equal(out["R"].cpu().numpy().view(np.uint32), ref["R"])
    np.testing.assert_array_equal(out["C"].cpu().numpy().view(np.uint32), ref["C"])
    steps = out["steps"].cpu().numpy()  # [graph][tree]
    np.testing.assert_array_equal(steps.sum(axis=0).astype(np.uint64), ref["steps"])
    lat = G.batch_latency_ms()
    assert lat.shape == (len(graphs),) and np.all(lat > 0)
    if kernel == 2:
        assert G.last_kernel() == bitmap + 1
    G.close()


def test_batch_farness_is_per_graph():
    graphs, alphas, u, offs = _batch(2)
    G = fc.Graph.batch(u, offs, alphas)
    tau = 400
    out = G.sample(5, tau)
    diag, far, clo = G.farness(out["R"], tau)
    d = diag.cpu().numpy()
    f = far.cpu().numpy()
    c = clo.cpu().numpy()
    for i, g in enumerate(graphs):
        a, b = offs[i], offs[i + 1]
        np.testing.assert_allclose(f[a:b], dense.farness_eq3(d[a:b]), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(c[a:b], dense.closeness(dense.farness_eq3(d[a:b])), rtol=1e-12)
        om = np.diag(dense.forest_matrix(g, alphas[i]))
        assert np.max(np.abs(d[a:b] - om)) < 0.15
    G.close()


def test_batch_rejects_edges_between_graphs():
    graphs, alphas, u, offs = _batch()
    su, sv, sw = u.edges()
    su = np.append(su, 0)
    sv = np.append(sv, offs[1])  # vertex 0 of graph 0 -- vertex 0 of graph 1
    sw = np.append(sw, np.float32(1.0))
    bad = synth.from_edges(u.n, su, sv, sw)
    with pytest.raises(fc.FcError) as e:
        fc.Graph.batch(bad, offs, alphas)
    assert e.value.status == fc.FC_EINVAL
