"""fc_forest_farness_noalloc: the allocation-free variant of fc_forest_farness.

Some callers cannot allocate device memory at the point where they need the
farness/closeness -- for example code running under a memory manager that
forbids allocations it does not make itself, or a serving loop whose device
memory is fixed once at start-up.  For them the library keeps the
combination's temporary per-block sums in a fixed device array compiled into
libfc.so (graphs up to 2^22 vertices).  These tests call both entry points
through the C ABI on the same inputs, twice in a row with different inputs
(the fixed array is shared by every call and keeps the last call's contents),
check that the results agree, compare them with the oracle's combination, and
run a graph of exactly 2^22 vertices, which uses every slot of the array.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import cv as ocv
from oracle import dense, native

pytestmark = pytest.mark.gpu

fc = pytest.importorskip("paper_2101_06192_gb300.fc")


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _run(entry, G, R, C, gp, x, tau):
    n = G.n
    outs = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = entry(G._h, 0, _p(R), _p(C), _p(gp), _p(x), int(tau), _p(outs[0]), _p(outs[1]), _p(outs[2]), stream)
    assert rc == fc.FC_OK, fc.lib().fc_last_error_message()
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def test_noalloc_matches_pool_version_on_two_calls_in_a_row():
    L = fc.lib()
    g = synth.barabasi_albert(50_000, 3, 5)
    G = fc.Graph.from_csr(g, [1.0])
    tau = 128
    x, _ = G.pivot_solve()
    gp = torch.from_numpy(np.random.default_rng(3).random(g.n).astype(np.float32)).cuda()
    runs = [G.sample(11, tau), G.sample(12, tau)]
    for variant in ("plain", "pivot", "cv"):
        for out in runs:  # two calls in a row, different inputs
            R = out["R"]
            C = out["C"] if variant == "cv" else None
            gpp = gp if variant == "cv" else None
            xp = x if variant == "pivot" else None
            ref = _run(L.fc_forest_farness, G, R, C, gpp, xp, tau)
            got = _run(L.fc_forest_farness_noalloc, G, R, C, gpp, xp, tau)
            for a, b in zip(got, ref):
                np.testing.assert_allclose(a, b, rtol=1e-9, atol=0)
    G.close()


def test_noalloc_inside_a_captured_cuda_graph():
    """The call launches kernels only (no allocation, no host read), so it can be
    captured: a CUDA graph holding fc_forest_farness_noalloc, replayed after new
    counts are written into its input buffer, gives the pool version's results
    at each replay."""
    L = fc.lib()
    g = synth.barabasi_albert(20_000, 3, 6)
    G = fc.Graph.from_csr(g, [1.0])
    tau = 64
    n = g.n
    G.sample(1, tau)  # warm-up outside the capture (launch shape, scratch)
    R = torch.zeros(n, dtype=torch.int32, device="cuda")
    outs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    cg = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(cg, stream=s):
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            rc = L.fc_forest_farness_noalloc(G._h, 0, _p(R), None, None, None, tau, _p(outs[0]), _p(outs[1]),
                                             _p(outs[2]), stream)
            assert rc == fc.FC_OK
    torch.cuda.current_stream().wait_stream(s)
    for sd in (21, 22):
        R.copy_(G.sample(sd, tau, with_C=False)["R"])
        cg.replay()
        torch.cuda.synchronize()
        ref = _run(L.fc_forest_farness, G, R, None, None, None, tau)
        for a, b in zip([o.cpu().numpy() for o in outs], ref):
            np.testing.assert_allclose(a, b, rtol=1e-9, atol=0)
    G.close()


def test_noalloc_rejects_graphs_beyond_its_capacity():
    L = fc.lib()
    n = (1 << 22) + 1
    G = fc.Graph(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), None, [1.0])
    R = torch.zeros(n, dtype=torch.int32, device="cuda")
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.fc_forest_farness_noalloc(G._h, 0, _p(R), None, None, None, 1, _p(d), None, None, stream)
    assert rc == fc.FC_EINVAL
    assert b"capacity" in L.fc_last_error_message()
    # the pool-backed entry point handles the same graph
    assert L.fc_forest_farness(G._h, 0, _p(R), None, None, None, 1, _p(d), None, None, stream) == fc.FC_OK
    torch.cuda.synchronize()
    G.close()


def test_noalloc_matches_oracle():
    """Plain, paper fill step (with the oracle's own pivot solution) and
    control-variate forms against the oracle's combination, Eq. 3 and Def. 2."""
    L = fc.lib()
    g = synth.erdos_renyi(1000, 8, 1)
    tau = 500
    G = fc.Graph.from_csr(g, [1.0])
    out = G.sample(31, tau)
    ref = native.wilson(g, 1.0, seed=31, tau=tau)
    assert np.array_equal(out["R"].cpu().numpy().view(np.uint32), ref["R"])
    p = ocv.p_root(g, 1.0)
    gp = np.random.default_rng(4).random(g.n).astype(np.float32)
    xo = dense.pivot_solution(g, 1.0)
    for variant in ("plain", "pivot", "cv"):
        C = out["C"] if variant == "cv" else None
        gpp = torch.from_numpy(gp).cuda() if variant == "cv" else None
        xp = torch.from_numpy(xo).cuda() if variant == "pivot" else None
        d, far, clo = _run(L.fc_forest_farness_noalloc, G, out["R"], C, gpp, xp, tau)
        if variant == "cv":
            exp = ocv.combine(ref["R"], ref["C"], tau, p, ocv.beta_from_prediction(gp.astype(np.float64), p))
        else:
            exp = dense.diag_from_counts(ref["R"], tau, xo if variant == "pivot" else None)
        np.testing.assert_allclose(d, exp, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(far, dense.farness_eq3(exp), rtol=1e-9)
        np.testing.assert_allclose(clo, dense.closeness(dense.farness_eq3(exp)), rtol=1e-9)
    G.close()


def test_noalloc_at_capacity_uses_every_slot():
    """n = 2^22 exactly: 16384 per-block sums plus the trace fill the array.
    Counts are given directly (no sampling), so the oracle's combination is
    cheap; two calls in a row with different counts."""
    L = fc.lib()
    n = 1 << 22
    # a cycle: every vertex has degree 2, so the control variate applies everywhere
    v = np.arange(n, dtype=np.int64)
    g = synth.from_edges(n, v, (v + 1) % n)
    G = fc.Graph.from_csr(g, [1.0])
    p = ocv.p_root(g, 1.0)
    rng = np.random.default_rng(9)
    tau = 64
    for call in range(2):
        R = rng.integers(0, tau + 1, n).astype(np.uint32)
        C = np.minimum(R, rng.integers(0, tau // 3, n).astype(np.uint32))
        gp = rng.random(n).astype(np.float32)
        Rt = torch.from_numpy(R.view(np.int32)).cuda()
        Ct = torch.from_numpy(C.view(np.int32)).cuda()
        gpt = torch.from_numpy(gp).cuda()
        got = _run(L.fc_forest_farness_noalloc, G, Rt, Ct, gpt, None, tau)
        pool = _run(L.fc_forest_farness, G, Rt, Ct, gpt, None, tau)
        exp = ocv.combine(R, C, tau, p, ocv.beta_from_prediction(gp.astype(np.float64), p))
        np.testing.assert_allclose(got[0], exp, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(got[1], dense.farness_eq3(exp), rtol=1e-9)
        for a, b in zip(got, pool):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
    G.close()
