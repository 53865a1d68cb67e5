"""Accuracy of the whole estimator at the benchmark size (BA n = 2^20, m = 8,
alpha = 1, tau = 1024 in one launch): diag(Omega) from the sampled trees against
CG columns on a degree-stratified reference set.

Theorem 1 (Hoeffding over tau independent trees) bounds each vertex's error
by sqrt(log(2/delta') / (2 tau)); with delta' = 1e-6 per vertex that is < 0.1
at tau = 1024, so the largest error over the reference set must stay below it.
The reference columns come from the library's multi-right-hand-side solver; since
the smallest eigenvalue of I + alpha L is at least 1, the error of each reference
entry is at most the residual norm |e_v - (I + alpha L) x_v|, which is
recomputed on the CPU in FP64 for a subset of the columns."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import cg as ocg

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _reference_vertices(g, count, seed):
    """Stratified by degree decile, plus the lowest-degree vertices (largest variance)."""
    rng = np.random.default_rng(seed)
    d = g.degrees()
    order = np.lexsort((np.arange(g.n), d))
    low = order[:count // 8]
    rest = order[count // 8:]
    deciles = np.array_split(rest, 10)
    per = (count - low.size) // 10
    picks = [low] + [rng.choice(b, size=min(per, b.size), replace=False) for b in deciles]
    return np.unique(np.concatenate(picks))


def test_ba_benchmark_size_estimate_within_hoeffding_bound():
    g = synth.barabasi_albert(1 << 20, 8, 2)
    tau = 1024
    G = fc.Graph.from_csr(g, [1.0])
    out = G.sample(31337, tau)
    diag, _, _ = G.farness(out["R"], tau)
    est = diag.cpu().numpy()
    vs = _reference_vertices(g, 512, 5)
    B = torch.zeros(vs.size, g.n, dtype=torch.float64, device="cuda")
    B[torch.arange(vs.size), torch.from_numpy(vs).cuda()] = 1.0
    X, _ = G.solve(B, rel_tol=1e-10)
    ref = X[torch.arange(vs.size), torch.from_numpy(vs).cuda()].cpu().numpy()
    # the reference's own error: residual norms in FP64 on the CPU
    A = ocg.system_matrix(g, 1.0)
    for j in range(0, vs.size, vs.size // 8):
        x = X[j].cpu().numpy()
        r = -(A @ x)
        r[vs[j]] += 1.0
        assert np.linalg.norm(r) <= 1e-7, (vs[j], np.linalg.norm(r))
    err = np.abs(est[vs] - ref)
    bound = math.sqrt(math.log(2.0 / 1e-6) / (2.0 * tau))
    assert bound < 0.1
    assert err.max() <= bound, (err.max(), bound)
    # and the errors look like sampling noise: mean squared error close to the
    # binomial variance Omega (1 - Omega) / tau, averaged over the reference set
    var = np.mean(ref * (1.0 - ref)) / tau
    assert np.mean(err ** 2) < 3.0 * var
    G.close()
