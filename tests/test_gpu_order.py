"""The trees are a function of the random stacks only (cycle popping): the GPU
sampler must give identical trees for every start order and launch shape,
including shapes that make its walkers collide often."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


@pytest.mark.parametrize("kind", ["ba", "grid", "grid_w", "er"])
def test_start_order_and_shape_invariance(kind):
    if kind == "ba":
        g, alphas, tau = synth.barabasi_albert(30_000, 4, 2), [1.0], 96
    elif kind == "grid":
        g, alphas, tau = synth.perturbed_grid(120, 100, 3, weighted=False), [0.1, 10.0], 48
    elif kind == "grid_w":
        g, alphas, tau = synth.perturbed_grid(90, 80, 7), [0.3, 8.0], 32
    else:
        g, alphas, tau = synth.erdos_renyi(2000, 3, 5), [2.0], 128
    G = fc.Graph.from_csr(g, alphas)
    ref = None
    kernels = (1, 2)
    for kernel in kernels:
        G.set_kernel(kernel)
        for order in ("degree", "degree_desc", "id", "id_desc", "auto"):
            for walkers, smem in ((0, 0), (1024, 1), (64, 1), (32, 0)):
                G.set_start_order(order)
                G.set_shape(walkers, 0, smem)
                out = G.sample(17, tau, want_parents=True, want_steps=True)
                cur = (out["parents"].cpu().numpy(), out["R"].cpu().numpy(), out["C"].cpu().numpy(),
                       out["steps"].cpu().numpy())
                if ref is None:
                    ref = cur
                else:
                    for x, y in zip(cur, ref):
                        np.testing.assert_array_equal(
                            x, y, err_msg=f"kernel={kernel} order={order} walkers={walkers} smem={smem}")
    G.close()
