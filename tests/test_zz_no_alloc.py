"""fc_forest_farness_noalloc: the allocation-free variant of fc_forest_farness.

Some callers cannot allocate device memory at the point where they need the
farness/closeness -- code running inside a CUDA graph capture, or under a
memory manager that forbids allocations it does not make itself.  For them the
library keeps the combination's temporary per-block sums in a fixed device
array compiled into libfc.so (graphs up to 2^22 vertices).  These tests call
both entry points through the C ABI on the same inputs, twice in a row with
different inputs (the fixed array is shared by every call and keeps the last
call's contents), and check that the results agree.  This file is collected
last so that a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

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
