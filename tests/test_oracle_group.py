"""Pins of the group forest closeness oracle (Sec. 5, Algorithm 3) against
definitions and closed forms that do not go through its rank-one updates."""
import itertools

import numpy as np
import pytest

import synth
from oracle import dense, group


def _weighted_er(n, deg, seed):
    g = synth.erdos_renyi(n, deg, seed)
    u, v, _ = g.edges()
    rng = np.random.default_rng(seed + 100)
    return synth.from_edges(n, u, v, rng.uniform(0.5, 3.0, u.size).astype(np.float32))


@pytest.mark.parametrize("alpha", [0.3, 1.0, 4.0])
def test_singleton_farness_is_electrical_farness_in_augmented_graph(alpha):
    # rho({v}) = tr((L*_{-v})^{-1}) is the electrical farness of v in G*: the
    # forest farness of Eq. 3 (sum over V) plus the resistance between v and
    # u*, which is Omega_vv (computed here from the forest matrix)
    g = _weighted_er(40, 5, 3)
    Om = dense.forest_matrix(g, alpha)
    far = dense.farness_eq3(np.diag(Om))
    for v in (0, 7, 19, 39):
        assert group.group_farness(g, alpha, [v]) == pytest.approx(far[v] + Om[v, v], rel=1e-10)


def test_greedy_choices_maximise_the_defined_gain():
    # every greedy step picks the vertex whose addition lowers rho(S) most,
    # each candidate evaluated by two dense inverses (no rank-one update)
    g = _weighted_er(12, 4, 5)
    for alpha in (0.5, 2.0):
        S, far = group.greedy(g, alpha, 5)
        Om = dense.forest_matrix(g, alpha)
        assert S[0] == int(np.argmin(np.diag(Om)))  # highest individual closeness
        for i in range(1, len(S)):
            gn = group.gains(g, alpha, S[:i])
            best = max(gn.values())
            assert gn[S[i]] == pytest.approx(best, rel=1e-12)
            assert gn[S[i]] > max(x for v, x in gn.items() if v != S[i]) - 1e-12
        for i in range(len(S)):
            assert far[i] == pytest.approx(group.group_farness(g, alpha, S[: i + 1]), rel=1e-10)


def test_group_farness_non_increasing_and_supermodular():
    # the Lemma of Sec. 5, checked on all nested pairs of small sets
    g = _weighted_er(9, 3, 8)
    alpha = 1.3
    rho = {}
    for r in range(0, 4):
        for S in itertools.combinations(range(9), r):
            if r:
                rho[S] = group.group_farness(g, alpha, S)
    for S in [s for s in rho if len(s) <= 2]:
        for T in [t for t in rho if len(t) == len(S) + 1 and set(S) <= set(t)]:
            assert rho[T] <= rho[S] + 1e-12
            if len(T) <= 2:
                for v in range(9):
                    if v in T:
                        continue
                    Sv, Tv = tuple(sorted(S + (v,))), tuple(sorted(T + (v,)))
                    assert rho[S] - rho[Sv] >= rho[T] - rho[Tv] - 1e-12


def test_edgeless_graph_closed_form_and_ties():
    # no edges: the remaining m vertices hang off u* alone, so
    # rho(S) = m + (m + 1) / |S| for every S; all vertices tie (rounding
    # decides which), so only the values and distinctness are fixed
    n = 10
    g = synth.from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64))
    S, far = group.greedy(g, 1.0, 4)
    assert len(set(S)) == 4 and all(0 <= v < n for v in S)
    for i, s in enumerate(range(1, 5)):
        m = n - s
        assert far[i] == pytest.approx(m + (m + 1) / s, rel=1e-12)


def test_star_centre_first():
    # a star with unit weights: the centre has the smallest Omega_vv
    n = 15
    g = synth.from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n))
    S, _ = group.greedy(g, 1.0, 1)
    assert S == [0]


def test_grounded_inverse_from_forest_matrix():
    # (L*_{-v})^{-1}[a, b] = Omega_ab - Omega_av - Omega_vb + Omega_vv with the
    # u* row of Omega read as zero: the identity the GPU path uses to form the
    # greedy's starting inverse from the forest matrix
    g = _weighted_er(30, 4, 11)
    alpha = 0.8
    n = g.n
    Ls = dense.augmented_laplacian(g, alpha)
    Om = np.zeros((n + 1, n + 1))
    Om[:n, :n] = dense.forest_matrix(g, alpha)
    for v in (0, 13):
        idx = [i for i in range(n + 1) if i != v]
        M = np.linalg.inv(Ls[np.ix_(idx, idx)])
        Mi = Om[np.ix_(idx, idx)] - Om[idx, v][:, None] - Om[v, idx][None, :] + Om[v, v]
        np.testing.assert_allclose(Mi, M, rtol=1e-10, atol=1e-12)


def test_greedy_guarantee_of_the_corollary():
    # Sec. 5, Corollary: rho({v0}) - rho(S) >= (1 - k / (e (k - 1))) (rho({v0}) - rho(S~))
    # for the greedy S of size k and the best S~ of size k (brute force)
    g = _weighted_er(9, 3, 17)
    for alpha, k in ((0.6, 3), (2.5, 4)):
        S, far = group.greedy(g, alpha, k)
        r0 = group.group_farness(g, alpha, [S[0]])
        best = min(group.group_farness(g, alpha, T) for T in itertools.combinations(range(9), k))
        bound = 1.0 - k / (np.e * (k - 1))
        assert r0 - far[-1] >= bound * (r0 - best) - 1e-12
        assert far[-1] >= best - 1e-12  # the greedy group is never better than the optimum


def test_against_exact_rationals():
    # tests/golden/group_exact.json: rho(S) for all S of size 1 and 2 and the
    # greedy sequence, in exact rational arithmetic (weights exact in FP32)
    import json
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "group_exact.json")
    with open(path) as f:
        cases = json.load(f)
    for c in cases:
        n = c["n"]
        u = np.array([e[0] for e in c["edges"]])
        v = np.array([e[1] for e in c["edges"]])
        w = np.array([float(Fraction(e[2])) for e in c["edges"]], dtype=np.float32)
        g = synth.from_edges(n, u, v, w)
        alpha = float(Fraction(c["alpha"]))
        for key, val in c["rho"].items():
            S = [int(x) for x in key.split(",")]
            assert group.group_farness(g, alpha, S) == pytest.approx(float(Fraction(val)), rel=1e-12)
        S, far = group.greedy(g, alpha, c["k"])
        assert S == c["greedy"]
        np.testing.assert_allclose(far, [float(Fraction(x)) for x in c["greedy_farness"]], rtol=1e-12)
