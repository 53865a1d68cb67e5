"""Pins of the oracle's Wilson sampler (Algorithm 2) and its random stacks."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.stats

import synth
from oracle import cv, dense, enumerate as enum, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

req = json.loads(sys.stdin.read())
ctr = torch.tensor(np.array(req["ctr"], dtype=np.uint32).view(np.int32))
out = torch.zeros_like(ctr)
_k[(1,)](ctr, out, req["seed"], len(req["ctr"]) // 4)
print(json.dumps(out.numpy().view(np.uint32).tolist()))
"""


def test_philox_matches_independent_library_implementation():
    """Philox4x32-10 (SC'11) of the oracle == triton.language.philox run by
    Triton's CPU interpreter (an independent published implementation), for
    counters with all four words in use and 64-bit keys."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = [2**32 - 1] * 4
    for seed in (0, 12345, 0xDEADBEEF12345678 >> 1):
        req = json.dumps({"ctr": ctr.ravel().tolist(), "seed": int(seed)})
        res = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=req, capture_output=True,
                             text=True, timeout=600, env={**os.environ, "TRITON_INTERPRET": "1"})
        assert res.returncode == 0, res.stderr[-2000:]
        ref = np.array(json.loads(res.stdout.strip().splitlines()[-1]), dtype=np.uint32).reshape(-1, 4)
        np.testing.assert_array_equal(native.philox(ctr, seed), ref)


def test_philox_uniformity():
    """Words are uniform: chi^2 of the top 8 bits of each word over 2^16 counters."""
    k = np.arange(1 << 16, dtype=np.uint32)
    ctr = np.stack([k, k * 0 + 3, k * 0 + 5, k * 0 + 1], axis=1)
    out = native.philox(ctr, 99)
    for j in range(4):
        h = np.bincount(out[:, j] >> 24, minlength=256)
        assert scipy.stats.chisquare(h).pvalue > 1e-4


@pytest.mark.parametrize("weighted,alpha", [(False, 0.8), (False, 1.0), (False, 6.0), (True, 0.8)])
def test_stack_entry_distribution(weighted, alpha):
    """One stack entry of v selects u* with prob 1/deg*(v) and neighbour j with
    alpha w_vj / deg*(v) (Sec. 4.1 edge weights of G*): chi^2 over 40k entries."""
    g = synth.random_small(6, 1.0, 3, weighted=weighted)  # K6
    v = 2
    K = 40000
    got = native.stack_entries(g, alpha, 7, 0, np.full(K, v), np.arange(K))
    nb = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
    w = np.ones(nb.size) if g.w is None else g.w[g.rowptr[v]:g.rowptr[v + 1]].astype(float)
    probs = np.concatenate([[1.0], alpha * w]) / (1.0 + alpha * w.sum())
    obs = np.array([np.sum(got == g.n)] + [np.sum(got == x) for x in nb])
    assert obs.sum() == K
    assert scipy.stats.chisquare(obs, probs * K).pvalue > 1e-4


def _parent_key(p):
    return np.ascontiguousarray(p, dtype=np.int32).tobytes()


@pytest.mark.parametrize("seed,weighted,alpha", [(21, False, 1.0), (24, False, 0.3), (22, True, 0.6), (23, True, 3.0)])
def test_tree_frequencies_match_matrix_tree_probabilities(seed, weighted, alpha):
    """Wilson's algorithm samples spanning trees of G* with probability
    proportional to the product of edge weights (uniform when unweighted):
    chi^2 of 60k sampled parent arrays against brute-force enumeration."""
    g = synth.random_small(4, 0.7, seed, weighted=weighted)
    dist, _ = enum.tree_distribution(g, alpha)
    tau = 60000
    out = native.wilson(g, alpha, seed=1000 + seed, tau=tau, want_parents=True)
    keys, counts = np.unique(out["parents"], axis=0, return_counts=True)
    got = {_parent_key(k): c for k, c in zip(keys, counts)}
    assert set(got) <= set(dist)  # every sample is a spanning tree of G*
    names = sorted(dist)
    obs = np.array([got.get(k, 0) for k in names], dtype=float)
    exp = np.array([dist[k] for k in names]) * tau
    # merge tiny-expectation cells so chi^2 is valid
    small = exp < 5
    if small.any():
        obs = np.concatenate([obs[~small], [obs[small].sum()]])
        exp = np.concatenate([exp[~small], [exp[small].sum()]])
    assert scipy.stats.chisquare(obs, exp).pvalue > 1e-4


def test_parents_form_spanning_trees_of_augmented_graph():
    g = synth.barabasi_albert(200, 3, 5, weighted=True)
    out = native.wilson(g, 1.5, seed=3, tau=20, want_parents=True)
    n = g.n
    adj = [set(g.colidx[g.rowptr[v]:g.rowptr[v + 1]].tolist()) for v in range(n)]
    for par in out["parents"]:
        for v in range(n):
            assert par[v] == n or par[v] in adj[v]
            x, hops = v, 0
            while x != n:
                x = par[x]
                hops += 1
                assert hops <= n


def test_prop1_unbiased_frequency():
    """Prop. 1: R[v]/tau is unbiased for r_{G*}(u*, v) = Omega_vv.  Per-vertex
    z-scores over tau = 20000 trees, Bonferroni over n = 40."""
    for weighted, alpha in ((False, 1.0), (True, 0.4)):
        g = synth.erdos_renyi(40, 4, 61, weighted=weighted)
        tau = 20000
        out = native.wilson(g, alpha, seed=11, tau=tau)
        om = np.diag(dense.forest_matrix(g, alpha))
        z = (out["R"] / tau - om) / np.sqrt(om * (1 - om) / tau + 1e-300)
        z[om >= 1 - 1e-15] = 0  # isolated vertices: R == tau exactly
        assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * g.n))
        iso = g.degrees() == 0
        assert np.all(out["R"][iso] == tau)


def test_order_invariance_bit_exact():
    """Random stacks make the tree a function of the stacks only (cycle popping):
    ascending-degree order, reversed order and a random order give identical
    parent arrays and identical step counts."""
    g = synth.barabasi_albert(300, 3, 71, weighted=True)
    a = native.wilson(g, 0.9, seed=5, tau=30, want_parents=True)
    rng = np.random.default_rng(1)
    for order in (np.arange(g.n)[::-1], rng.permutation(g.n)):
        b = native.wilson(g, 0.9, seed=5, tau=30, order=order, want_parents=True)
        np.testing.assert_array_equal(a["parents"], b["parents"])
        np.testing.assert_array_equal(a["steps"], b["steps"])
        np.testing.assert_array_equal(a["R"], b["R"])


def test_expected_departures_equal_sum_deg_star_omega():
    """Expected departures per tree = sum_v deg*(v) Omega_vv (mean number of
    visits of v before absorption at u*; bounded by alpha vol + n as in Prop. 3)."""
    g = synth.erdos_renyi(60, 6, 81, weighted=True)
    alpha = 2.0
    tau = 8000
    out = native.wilson(g, alpha, seed=13, tau=tau)
    om = np.diag(dense.forest_matrix(g, alpha))
    dw = np.diag(dense.laplacian(g))
    pred = np.sum((1 + alpha * dw) * om)
    s = out["steps"].astype(float)
    z = (s.mean() - pred) / (s.std(ddof=1) / math.sqrt(tau))
    assert abs(z) < 4.5
    assert pred <= alpha * dw.sum() + g.n


def test_visits_per_vertex_equal_deg_star_omega():
    """Departures from v per tree of G* have mean deg*(v) Omega_vv (visits of a
    walk killed at u*): per-vertex z-scores over 3000 trees; totals = steps."""
    g = synth.erdos_renyi(40, 4, 17, weighted=True)
    alpha = 0.7
    T = 3000
    K = np.stack([native.wilson(g, alpha, seed=4, tau=1, tree_offset=t, want_C=False, want_visits=True)["visits"]
                  for t in range(T)]).astype(np.float64)
    tot = native.wilson(g, alpha, seed=4, tau=T, want_C=False, want_visits=True)
    assert int(tot["visits"].sum()) == int(tot["steps"].sum())
    om = np.diag(dense.forest_matrix(g, alpha))
    dstar = 1.0 + alpha * np.array([g.w[g.rowptr[v]:g.rowptr[v + 1]].astype(np.float64).sum() for v in range(g.n)])
    z = (K.mean(axis=0) - dstar * om) / (K.std(axis=0, ddof=1) / math.sqrt(T) + 1e-300)
    z[K.std(axis=0) == 0] = 0
    assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * g.n))
    # the visit estimate of diag(Omega), with deg* summed as the builder does
    np.testing.assert_allclose(dense.deg_star(g, alpha), dstar, rtol=1e-15)
    est = dense.diag_from_visits(tot["visits"], T, dense.deg_star(g, alpha))
    np.testing.assert_allclose(est, (K / dstar).mean(axis=0), rtol=1e-12)
    # much smaller per-tree variance than Prop. 1's indicator on this graph
    X = np.stack([native.wilson(g, alpha, seed=4, tau=1, tree_offset=t, want_C=False)["R"] for t in range(T)])
    assert (K / dstar).var(axis=0).mean() < 0.2 * X.astype(np.float64).var(axis=0).mean()


def test_tree_offset_additivity():
    """Trees are indexed globally: sampling [0, a) and [a, a+b) separately gives the
    same counts as [0, a+b) (resume / sharding identity)."""
    g = synth.erdos_renyi(120, 5, 91)
    full = native.wilson(g, 1.0, seed=17, tau=50, want_parents=True)
    p1 = native.wilson(g, 1.0, seed=17, tau=20, want_parents=True)
    p2 = native.wilson(g, 1.0, seed=17, tau=30, tree_offset=20, want_parents=True)
    np.testing.assert_array_equal(full["R"], p1["R"] + p2["R"])
    np.testing.assert_array_equal(full["C"], p1["C"] + p2["C"])
    np.testing.assert_array_equal(full["parents"], np.concatenate([p1["parents"], p2["parents"]]))


def test_control_variate_counts():
    """C_t(v) = [stack entry 0 of v selects u*]: C = 1 forces parent u*, and the
    frequency of C matches the exact p_v (z-test)."""
    g = synth.barabasi_albert(100, 2, 7, weighted=False)
    for t in range(10):
        o = native.wilson(g, 1.0, seed=23, tau=1, tree_offset=t, want_parents=True)
        assert np.all(o["parents"][0][o["C"] == 1] == g.n)
        first = native.stack_entries(g, 1.0, 23, t, np.arange(g.n), np.zeros(g.n))
        np.testing.assert_array_equal(o["C"], (first == g.n).astype(np.uint32))
    tau = 20000
    o = native.wilson(g, 1.0, seed=29, tau=tau)
    p = cv.p_root(g, 1.0)
    z = (o["C"] / tau - p) / np.sqrt(p * (1 - p) / tau)
    assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * g.n))


def test_p_root_exact_probabilities():
    """The exact 53-bit count of the u*-decision is within 2^-52 of 1/deg*(v)
    (deg* = 1 + alpha d unweighted, 1 + alpha d_w weighted), and is the smallest
    u53 whose scaled value reaches 1 (checked at the boundary)."""
    for d, alpha in ((0, 1.0), (1, 1.0), (7, 0.1), (100, 3.3), (12345, 1.0)):
        p = native.p_root(d, alpha, 0.0, False)
        assert abs(p - 1.0 / (1.0 + alpha * d)) <= 2**-52
        t = 1.0 + alpha * d
        u = int(round(p * 2**53))
        assert u == 2**53 or (u * 2.0**-53) * t >= 1.0
        assert u == 0 or ((u - 1) * 2.0**-53) * t < 1.0
    for d, alpha, S in ((1, 1.0, 3.5), (4, 0.1, 22.0), (9, 10.0, 50.25), (0, 2.0, 0.0)):
        p = native.p_root(d, alpha, S, True)
        assert abs(p - 1.0 / (1.0 + alpha * S)) <= 2**-52
    g = synth.random_small(6, 1.0, 4, weighted=True)
    p = cv.p_root(g, 0.5)
    S = native.row_prefix(g)
    for v in range(g.n):
        assert abs(p[v] - 1 / (1 + 0.5 * S[g.rowptr[v + 1] - 1])) <= 2**-52


def test_control_variate_unbiased_any_prediction():
    """The CV estimator is unbiased for any beta (E[C] = p_v exactly), and at the
    true Omega its per-tree variance is (1 - Omega)(Omega - p)/(1 - p)."""
    g = synth.erdos_renyi(30, 3, 33)
    alpha = 1.0
    om = np.diag(dense.forest_matrix(g, alpha))
    p = cv.p_root(g, alpha)
    T = 4000
    X = np.zeros((T, g.n))
    Cm = np.zeros((T, g.n))
    for t in range(T):
        o = native.wilson(g, alpha, seed=41, tau=1, tree_offset=t, want_steps=False)
        X[t] = o["R"]
        Cm[t] = o["C"]
    nonfinite = np.where(np.arange(g.n) % 3 == 0, np.nan, np.where(np.arange(g.n) % 3 == 1, np.inf, -np.inf))
    for gp in (np.zeros(g.n), om, np.random.default_rng(0).random(g.n), nonfinite):
        beta = cv.beta_from_prediction(gp, p)
        Y = X - beta * (Cm - p)
        z = (Y.mean(axis=0) - om) / (Y.std(axis=0, ddof=1) / math.sqrt(T) + 1e-12)
        z[om >= 1 - 1e-15] = 0
        assert np.max(np.abs(z)) < scipy.stats.norm.isf(1e-4 / (2 * g.n))
    beta = cv.beta_from_prediction(om, p)
    Y = X - beta * (Cm - p)
    ok = om < 1 - 1e-12
    var_pred = (1 - om[ok]) * (om[ok] - p[ok]) / (1 - p[ok])
    ratio = Y.var(axis=0, ddof=1)[ok] / var_pred
    assert 0.85 < np.mean(ratio) < 1.15
    assert np.mean(Y.var(axis=0)[ok]) < np.mean(X.var(axis=0)[ok])
    # plain estimator's combination via Algorithm 1's fill step == R/tau
    R = X.sum(axis=0)
    np.testing.assert_allclose(cv.combine(R, Cm.sum(axis=0), T, p, np.zeros(g.n)), R / T)


def test_beta_of_nonfinite_predictions():
    """clip(g, p, 1) on predictions that are not finite: -inf and NaN give p
    (beta = 1, the full control variate), +inf gives 1 (beta = 0, the plain
    estimator); a vertex with p = 1 (isolated) always gets beta = 0."""
    p = np.array([0.2, 0.2, 0.2, 0.5, 1.0])
    gp = np.array([np.nan, np.inf, -np.inf, 0.75, np.nan])
    np.testing.assert_array_equal(cv.beta_from_prediction(gp, p), [1.0, 0.0, 1.0, 0.5, 0.0])


def test_hoeffding_failure_rate():
    """Thm. 1: with tau from Algorithm 1 the max-abs error exceeds eps with
    probability at most delta (here: over 40 independent seeds)."""
    g = synth.erdos_renyi(30, 4, 51)
    alpha, eps, delta, kappa = 1.0, 0.2, 0.2, 0.5
    tau = dense.tau_for(eps, delta, kappa, g.m)
    om = np.diag(dense.forest_matrix(g, alpha))
    fails = 0
    seeds = 40
    for s in range(seeds):
        o = native.wilson(g, alpha, seed=500 + s, tau=tau, want_C=False, want_steps=False)
        fails += np.max(np.abs(o["R"] / tau - om)) > eps
    assert fails <= delta * seeds


def test_row_prefix_exact_for_grid_weights():
    """Per-row FP64 prefix of FP32 weights in [1, 10] is exact (sums of < 2^24
    multiples of 2^-23), hence equal to numpy's cumulative sum."""
    g = synth.perturbed_grid(40, 30, 5)
    S = native.row_prefix(g)
    for v in (0, 17, 600, g.n - 1):
        a, b = g.rowptr[v], g.rowptr[v + 1]
        np.testing.assert_array_equal(S[a:b], np.cumsum(g.w[a:b].astype(np.float64)))
