"""The sampling launch and the per-alpha combinations captured into one CUDA
graph give the same results as direct calls, on every replay."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def test_captured_multi_alpha_step_replays_exactly():
    g = synth.perturbed_grid(64, 48, 3)
    alphas = [0.1, 1.0, 10.0]
    tau = 32
    G = fc.Graph.from_csr(g, alphas)
    ref = G.sample(77, tau)  # uncaptured call: also sizes the sampler scratch
    ref_d = [G.farness(ref["R"], tau, alpha_idx=a)[0].clone() for a in range(3)]
    s = torch.cuda.Stream()
    R = torch.zeros(3 * g.n, dtype=torch.int32, device="cuda")
    C = torch.zeros(3 * g.n, dtype=torch.int32, device="cuda")
    diag = [torch.empty(g.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            R.zero_()
            C.zero_()
            G.sample_async(77, tau, R, C, stream=s)
            for a in range(3):
                d, _, _ = G.farness(R, tau, alpha_idx=a, stream=s)
                diag[a].copy_(d)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        G.check()
        assert torch.equal(R, ref["R"]) and torch.equal(C, ref["C"])
        for a in range(3):
            np.testing.assert_array_equal(diag[a].cpu().numpy(), ref_d[a].cpu().numpy())
    G.close()
