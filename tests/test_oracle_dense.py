"""Pins of the oracle's dense routines against facts the paper and the
mathematics fix (not against the oracle itself)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import cg, dense, enumerate as enum, exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "omega_exact.json")


def _graph_from_golden(case):
    n = case["n"]
    u = [e[0] for e in case["edges"]]
    v = [e[1] for e in case["edges"]]
    w = [float(Fraction(e[2])) for e in case["edges"]]
    return synth.from_edges(n, u, v, w)


@pytest.mark.parametrize("case", json.load(open(GOLDEN)), ids=lambda c: c["name"])
def test_forest_matrix_matches_exact_rationals(case):
    """Golden: exact Omega from Gauss-Jordan over Fractions == matrix-forest
    enumeration (written by tests/golden/make_golden.py).  Sec. 2, Eq. 3."""
    g = _graph_from_golden(case)
    alpha = float(Fraction(case["alpha"]))
    Om = dense.forest_matrix(g, alpha)
    ref = np.array([[float(Fraction(x)) for x in row] for row in case["omega"]])
    np.testing.assert_allclose(Om, ref, rtol=0, atol=1e-14)
    far = dense.farness_eq3(np.diag(Om))
    np.testing.assert_allclose(far, [float(Fraction(x)) for x in case["farness_eq3"]], atol=1e-13)
    M = alpha * dense.laplacian(g) + np.eye(g.n)
    assert math.isclose(np.linalg.det(M), float(Fraction(case["det_I_plus_alphaL"])), rel_tol=1e-12)


@pytest.mark.parametrize("seed,weighted", [(1, False), (2, True), (3, True)])
def test_invariants_doubly_stochastic_symmetric(seed, weighted):
    """Omega 1 = 1 (Sec. 4.2, doubly stochastic), Omega symmetric, 0 < Omega_vv <= 1,
    and Omega_vv >= 1 / (1 + alpha d_w(v)) ((A^-1)_ii >= 1/A_ii for SPD A)."""
    g = synth.erdos_renyi(60, 5, seed, weighted=weighted)
    for alpha in (0.1, 1.0, 7.5):
        Om = dense.forest_matrix(g, alpha)
        np.testing.assert_allclose(Om.sum(axis=1), 1.0, atol=1e-12)
        np.testing.assert_allclose(Om, Om.T, atol=1e-13)
        d = np.diag(Om)
        assert np.all(d > 0) and np.all(d <= 1 + 1e-15)
        dw = np.diag(dense.laplacian(g))
        assert np.all(d >= 1.0 / (1.0 + alpha * dw) - 1e-14)


def test_closed_forms_empty_K2_Kn():
    """No edges: Omega = I.  K_n: Omega_vv = (1 + alpha) / (1 + alpha n)
    (eigenvalues of L_Kn are 0 and n, Omega = J/n + (I - J/n)/(1 + alpha n))."""
    np.testing.assert_allclose(dense.forest_matrix(synth.empty(5), 3.0), np.eye(5), atol=0)
    for n in (2, 3, 7, 20):
        for alpha in (0.25, 1.0, 4.0):
            d = np.diag(dense.forest_matrix(synth.complete(n), alpha))
            np.testing.assert_allclose(d, (1 + alpha) / (1 + alpha * n), rtol=1e-13)


@pytest.mark.parametrize("N,wt", [(5, None), (12, 2.5), (31, None)])
def test_closed_form_cycle(N, wt):
    """Cycle C_N: Laplacian eigenvalues 2w(1 - cos(2 pi k / N)); the diagonal of
    Omega is constant and equals the mean of 1 / (1 + alpha lambda_k)."""
    w = 1.0 if wt is None else wt
    for alpha in (0.5, 3.0):
        lam = 2 * w * (1 - np.cos(2 * np.pi * np.arange(N) / N))
        ref = np.mean(1.0 / (1.0 + alpha * lam))
        d = np.diag(dense.forest_matrix(synth.cycle(N, wt), alpha))
        np.testing.assert_allclose(d, ref, rtol=1e-12)


def test_closed_form_torus_dense_and_cg():
    """W x H torus: eigenvalues w (4 - 2 cos(2 pi i / W) - 2 cos(2 pi j / H)).
    Dense inverse at 8x6 and the FP64 CG ground truth at 64x48."""
    for (W, H, use_cg) in ((8, 6, False), (64, 48, True)):
        g = synth.torus(W, H, 1.5)
        alpha = 2.0
        i = np.arange(W)[:, None]
        j = np.arange(H)[None, :]
        lam = 1.5 * (4 - 2 * np.cos(2 * np.pi * i / W) - 2 * np.cos(2 * np.pi * j / H))
        ref = np.mean(1.0 / (1.0 + alpha * lam))
        if use_cg:
            d = cg.omega_diag_at(g, alpha, [0, 17, W * H - 1])
        else:
            d = np.diag(dense.forest_matrix(g, alpha))
        np.testing.assert_allclose(d, ref, rtol=1e-10)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_matrix_forest_theorem_bruteforce(seed):
    """Omega[u, v] = weighted share of spanning trees of G* whose path from v
    enters u* through u (Sec. 2 matrix-forest theorem); total weight =
    det(I + alpha L) (Kirchhoff)."""
    g = synth.random_small(5, 0.6, seed, weighted=True)
    alpha = 0.7
    Om = dense.forest_matrix(g, alpha)
    np.testing.assert_allclose(enum.omega_by_forests(g, alpha), Om, atol=1e-12)
    _, total = enum.tree_distribution(g, alpha)
    M = alpha * dense.laplacian(g) + np.eye(g.n)
    assert math.isclose(total, np.linalg.det(M), rel_tol=1e-12)


def test_farness_eq3_equals_definition2():
    """Eq. 3 (diagonal + trace) equals Def. 2 (sum of Eq. 1 distances)."""
    for seed, weighted in ((4, False), (5, True)):
        g = synth.barabasi_albert(80, 3, seed, weighted=weighted)
        Om = dense.forest_matrix(g, 1.3)
        np.testing.assert_allclose(dense.farness_eq3(np.diag(Om)), dense.farness_def2(Om), rtol=1e-12)
        c = dense.closeness(dense.farness_def2(Om))
        assert np.all(c > 0)


def test_effective_resistance_to_pivot_is_omega_diag():
    """Prop. 2 with v2 = u*: r_{G*}(u*, v) = Omega_vv, computed from the
    pseudo-inverse of L* (Eq. 2) -- the quantity Prop. 1's frequency estimates."""
    g = synth.erdos_renyi(40, 4, 21, weighted=True)
    alpha = 0.9
    P = dense.augmented_pinv(g, alpha)
    # library cross-check of the pseudo-inverse (the paper checks against NumPy pinv)
    np.testing.assert_allclose(P, np.linalg.pinv(dense.augmented_laplacian(g, alpha), rcond=1e-10),
                               atol=1e-11)
    n = g.n
    r = P[n, n] + np.diag(P)[:n] - 2 * P[:n, n]
    np.testing.assert_allclose(r, np.diag(dense.forest_matrix(g, alpha)), atol=1e-11)
    # Prop. 2 for a pair inside V: forest distance == effective resistance in G*
    Om = dense.forest_matrix(g, alpha)
    rho = dense.forest_distance(Om)
    r_pair = P[3, 3] + P[7, 7] - 2 * P[3, 7]
    assert abs(rho[3, 7] - r_pair) < 1e-11


def test_pivot_solve_closed_form_and_fill_step_reading():
    """Algorithm 1's pivot solve: x(v) - x(u*) = -1/(n+1) for every v (the
    right-hand side restricted to V is a multiple of 1, an eigenvector of
    I + alpha L with eigenvalue 1), |x|_inf <= 2 (proof of Thm. 1), and
    (L*^+)[V, V] = Omega - ((n+2)/(n+1)^2) J, so the fill step with exact counts
    R = tau Omega_vv plus the block offset returns Omega_vv."""
    for seed in (31, 32):
        g = synth.erdos_renyi(35, 4, seed, weighted=True)
        alpha = 1.7
        n = g.n
        x = dense.pivot_solution(g, alpha)
        np.testing.assert_allclose(x[:n] - x[n], -1.0 / (n + 1), atol=1e-13)
        assert np.max(np.abs(x)) <= 2.0
        assert abs(x.sum()) < 1e-12  # mean-zero (pseudo-inverse) gauge
        Om = dense.forest_matrix(g, alpha)
        P = np.linalg.pinv(dense.augmented_laplacian(g, alpha), rcond=1e-10)
        np.testing.assert_allclose(P[:n, :n], Om - dense.pinv_block_offset(n), atol=1e-12)
        tau = 1000
        R = tau * np.diag(Om)  # fractional "counts": checks the arithmetic only
        lit = dense.combine_fill_step(R, tau, x)
        np.testing.assert_allclose(lit, np.diag(P)[:n], atol=1e-12)
        np.testing.assert_allclose(dense.diag_from_counts(R, tau, x), np.diag(Om), atol=1e-12)


def test_tau_is_minimal_hoeffding_union_bound():
    """tau of Algorithm 1 is the least integer with 2 m exp(-2 tau eps'^2) <= delta,
    eps' = (1 - kappa) eps (Hoeffding + union bound, proof of Thm. 1)."""
    for eps, delta, kappa, m in ((0.1, 0.1, 0.5, 60), (0.05, 1e-3, 0.3, 10**6), (0.3, 0.5, 0.9, 17)):
        t = dense.tau_for(eps, delta, kappa, m)
        ep = (1 - kappa) * eps
        assert 2 * m * math.exp(-2 * t * ep * ep) <= delta * (1 + 1e-12)
        assert 2 * m * math.exp(-2 * (t - 1) * ep * ep) > delta


def test_eta_bound_gives_kappa_eps_over_3():
    """eta * sqrt(alpha (c+2) vol) * 2 = kappa eps / 3 (proof of Thm. 1)."""
    eps, kappa, alpha, n, vol = 0.1, 0.5, 1.0, 1000, 8000.0
    eta = dense.eta_for(eps, kappa, alpha, n, vol)
    c = n / (alpha * vol)
    assert math.isclose(eta * math.sqrt(alpha * (c + 2) * vol) * 2, kappa * eps / 3, rel_tol=1e-12)


def _max_over_sign_vectors(M):
    """max of x^T M x over x in {-1, +1}^n (brute force; x and -x agree)."""
    n = M.shape[0]
    best = -np.inf
    for bits in range(2 ** (n - 1)):
        x = np.array([1.0 if (bits >> i) & 1 else -1.0 for i in range(n - 1)] + [1.0])
        best = max(best, float(x @ M @ x))
    return best


def _bipartite_weighted_grid():
    rng = np.random.default_rng(5)
    u, v = [], []
    for r in range(3):
        for c in range(4):
            i = 4 * r + c
            if c < 3:
                u.append(i), v.append(i + 1)
            if r < 2:
                u.append(i), v.append(i + 4)
    return synth.from_edges(12, u, v, rng.uniform(0.5, 3.0, len(u)))


@pytest.mark.parametrize("name,g,bipartite", [
    ("cycle8", synth.cycle(8), True),
    ("path7", synth.path(7), True),
    ("grid3x4_weighted", _bipartite_weighted_grid(), True),
    ("cycle9", synth.cycle(9), False),
    ("complete6", synth.complete(6), False),
    ("er11", synth.random_small(11, 0.4, 3, True), False),
])
@pytest.mark.parametrize("alpha", [0.3, 2.0])
def test_eta_against_the_tight_norm_equivalence(name, g, bipartite, alpha):
    """Proof of Thm. 1: with L' = alpha L + I and c = n / (alpha vol), every x has
    ||x||_inf <= ||x||_{L'} <= sqrt(alpha (c + 2) vol) ||x||_inf, and eta makes the
    solver's max-norm error eta sqrt(alpha (c + 2) vol) ||x||_inf <= kappa eps / 3 for
    ||x||_inf <= 2.  The upper constant is checked here as what it is, the maximum
    of x^T L' x over the cube (a convex function peaks at a vertex, so at a sign
    vector), found by brute force: equal to alpha (c + 2) vol on bipartite graphs
    (x the 2-colouring: every edge term is 4 w), below it otherwise; the lower one
    as the smallest eigenvalue of L' (= 1).  eta is then pinned by that maximum,
    not by its own formula."""
    n = g.n
    Lp = alpha * dense.laplacian(g) + np.eye(n)
    vol = float(dense.laplacian(g).trace())  # sum of weighted degrees
    top = _max_over_sign_vectors(Lp)
    c = n / (alpha * vol)
    if bipartite:
        assert math.isclose(top, alpha * (c + 2) * vol, rel_tol=1e-12)
    else:
        assert top < alpha * (c + 2) * vol * (1 - 1e-9)
    assert math.isclose(float(np.linalg.eigvalsh(Lp)[0]), 1.0, rel_tol=0, abs_tol=1e-12)
    eps, kappa = 0.1, 0.5
    eta = dense.eta_for(eps, kappa, alpha, n, vol)
    worst = eta * math.sqrt(top) * 2.0  # ||x||_inf = 2, the proof's bound on x
    if bipartite:
        assert math.isclose(worst, kappa * eps / 3, rel_tol=1e-12)
    else:
        assert worst < kappa * eps / 3
    # a relative L'-norm error of eta, in the direction that maximises the max
    # norm, stays within that budget (max over unit-L'-norm e of |e_i| is
    # sqrt((L'^-1)_ii), Cauchy-Schwarz)
    x = dense.pivot_solution(g, alpha)[:n]
    x_norm = math.sqrt(float(x @ Lp @ x))
    e_inf = eta * x_norm * math.sqrt(float(np.max(np.diag(np.linalg.inv(Lp)))))
    assert e_inf <= kappa * eps / 3 * float(np.max(np.abs(x))) / 2.0 + 1e-15


def test_top_k_ties_and_order():
    d = np.array([0.3, 0.1, 0.2, 0.1, 0.5])
    assert dense.top_k(d, 3).tolist() == [1, 3, 2]
    far = dense.farness_eq3(d)
    assert dense.top_k(d, 5).tolist() == sorted(range(5), key=lambda i: (far[i], i))


def test_cg_matches_dense_columns():
    """The FP64 CG ground truth (Sec. 6.1) agrees with the dense inverse."""
    g = synth.barabasi_albert(300, 4, 41, weighted=True)
    alpha = 3.0
    Om = dense.forest_matrix(g, alpha)
    vs = [0, 5, 299, 150]
    X = cg.omega_columns(g, alpha, vs)
    np.testing.assert_allclose(X, Om[:, vs], atol=1e-10)
