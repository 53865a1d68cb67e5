"""Dense FP64 definitions of the quantities the method estimates (test
infrastructure only; never called by the product path).

Everything is the plain definition written out with numpy/scipy primitives:
  * Laplacian L = diag(deg_w) - A_w                       (Sec. 2, Definitions)
  * forest matrix Omega = (alpha L + I)^{-1}               (Sec. 2, "Forest Distance")
  * pairwise forest distance rho(u, v)                     (Def. 1, Eq. 1)
  * forest farness rho(u) = sum_{v != u} rho(u, v)         (Def. 2)
  * farness from the diagonal, rho(v) = n Omega_vv + tr Omega - 2   (Eq. 3)
  * forest closeness n / rho(u)                            (Def. 2)
  * ranking: top vertices have the lowest Omega_vv         (Sec. 6.1, footnote)
  * Algorithm 1 parameters eta and tau (its solver-accuracy and sample-size steps)
  * Algorithm 1's pivot solve L* x = e_{u*} - 1/(n+1) 1 and its combination step
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def adjacency(g) -> np.ndarray:
    A = np.zeros((g.n, g.n), dtype=np.float64)
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    A[src, g.colidx] = w
    return A


def laplacian(g) -> np.ndarray:
    """L = diag(deg_G) - A_G with weighted degrees (Sec. 2)."""
    A = adjacency(g)
    return np.diag(A.sum(axis=1)) - A


def forest_matrix(g, alpha: float) -> np.ndarray:
    """Omega_alpha = (alpha L + I)^{-1} by a dense Cholesky factorisation (Sec. 2)."""
    M = alpha * laplacian(g) + np.eye(g.n)
    c = scipy.linalg.cho_factor(M, lower=True)
    return scipy.linalg.cho_solve(c, np.eye(g.n))


def augmented_laplacian(g, alpha: float) -> np.ndarray:
    """Laplacian of G* (Sec. 4.1): edges of G scaled by alpha, every vertex joined
    to the universal vertex u* (index n) by an edge of weight 1."""
    n = g.n
    Ls = np.zeros((n + 1, n + 1))
    Ls[:n, :n] = alpha * laplacian(g) + np.eye(n)
    Ls[:n, n] = -1.0
    Ls[n, :n] = -1.0
    Ls[n, n] = n
    return Ls


def forest_distance(Omega: np.ndarray) -> np.ndarray:
    """rho(u, v) = Omega_uu + Omega_vv - 2 Omega_uv (Def. 1, Eq. 1)."""
    d = np.diag(Omega)
    return d[:, None] + d[None, :] - 2.0 * Omega


def farness_def2(Omega: np.ndarray) -> np.ndarray:
    """rho(u) = sum over v != u of rho(u, v) (Def. 2); the v = u term is zero."""
    return forest_distance(Omega).sum(axis=1)


def farness_eq3(diag: np.ndarray, trace: float | None = None) -> np.ndarray:
    """rho(v) = n Omega_vv + tr(Omega) - 2 (Eq. 3, Omega doubly stochastic)."""
    n = diag.size
    tr = float(np.sum(diag)) if trace is None else trace
    return n * diag + tr - 2.0


def closeness(farness: np.ndarray) -> np.ndarray:
    """Forest closeness n / rho(u) (Def. 2)."""
    n = farness.size
    with np.errstate(divide="ignore"):
        return n / farness


def top_k(diag: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k most central vertices: ascending Omega_vv (= ascending
    farness by Eq. 3), ties broken by ascending vertex id."""
    order = np.lexsort((np.arange(diag.size), diag))
    return order[:k].astype(np.int32)


def tau_for(eps: float, delta: float, kappa: float, m: int) -> int:
    """Number of trees of Algorithm 1: ceil(log(2m/delta) / (2 (1-kappa)^2 eps^2)),
    natural logarithm (Hoeffding's bound, proof of Thm. 1)."""
    return int(math.ceil(math.log(2.0 * m / delta) / (2.0 * (1.0 - kappa) ** 2 * eps ** 2)))


def eta_for(eps: float, kappa: float, alpha: float, n: int, vol: float) -> float:
    """Solver accuracy of Algorithm 1: kappa eps / (6 sqrt(alpha (c + 2) vol)),
    c = n / (alpha vol)."""
    c = n / (alpha * vol)
    return kappa * eps / (6.0 * math.sqrt(alpha * (c + 2.0) * vol))


def augmented_pinv(g, alpha: float) -> np.ndarray:
    """Moore-Penrose pseudo-inverse of L*.  G* is connected (u* is adjacent to
    every vertex), so its Laplacian has the one-dimensional kernel span(1) and
    L*^+ = (L* + J/(n+1))^{-1} - J/(n+1)."""
    n1 = g.n + 1
    Ls = augmented_laplacian(g, alpha)
    J = np.full((n1, n1), 1.0 / n1)
    return np.linalg.inv(Ls + J) - J


def pivot_solution(g, alpha: float) -> np.ndarray:
    """Algorithm 1's pivot solve: the minimum-norm (mean-zero) solution of
    L* x = e_{u*} - 1/(n+1) 1 on G*, i.e. x = L*^+ (e_{u*} - 1/(n+1) 1).
    Returns x of length n+1, x[n] = x(u*)."""
    n = g.n
    b = -np.full(n + 1, 1.0 / (n + 1))
    b[n] += 1.0
    return augmented_pinv(g, alpha) @ b


def combine_fill_step(R: np.ndarray, tau: int, x: np.ndarray) -> np.ndarray:
    """Algorithm 1's fill step taken literally: R[v]/tau - x(u*) + 2 x(v).
    With x = L*^+ e_{u*} this is the estimate of diag(L*^+) restricted to V."""
    n = R.size
    return R.astype(np.float64) / tau - x[n] + 2.0 * x[:n]


def pinv_block_offset(n: int) -> float:
    """(L*^+)[V, V] = Omega - ((n+2)/(n+1)^2) J  (exact identity for G*; the paper's
    block claim in Sec. 4.1 omits this rank-one shift)."""
    return (n + 2.0) / (n + 1.0) ** 2


def diag_from_counts(R: np.ndarray, tau: int, x: np.ndarray | None = None) -> np.ndarray:
    """diag(Omega) estimate used throughout: the fill step of Algorithm 1 followed by
    the block correction; equals R/tau whenever x is the exact pivot solution.
    Without x the estimate is R/tau directly (Prop. 1: unbiased for
    r_{G*}(u*, v) = Omega_vv)."""
    if x is None:
        return R.astype(np.float64) / tau
    return combine_fill_step(R, tau, x) + pinv_block_offset(R.size)


def deg_star(g, alpha) -> np.ndarray:
    """deg*(v) = fl(1 + fl(alpha d_w(v))) with d_w(v) the row's FP32 weights
    summed left to right in FP64 (alpha a float or a per-vertex array)."""
    dw = np.zeros(g.n)
    for v in range(g.n):
        s = 0.0
        for e in range(g.rowptr[v], g.rowptr[v + 1]):
            s = s + (1.0 if g.w is None else float(g.w[e]))
        dw[v] = s
    return 1.0 + np.asarray(alpha, dtype=np.float64) * dw


def diag_from_visits(visits: np.ndarray, tau: int, dstar: np.ndarray) -> np.ndarray:
    """Visit estimate of diag(Omega) (not in the paper).  In Wilson's algorithm
    on G* the departures K_v from v in one tree do not depend on the start
    order; with v as the first start vertex they are the visits to v of a walk
    from v killed at u*, whose mean is the Green's function deg*(v) r_{G*}(u*, v)
    = deg*(v) Omega_vv.  So visits[v] / (tau deg*(v)) is unbiased for Omega_vv."""
    return visits.astype(np.float64) / (float(tau) * dstar)
