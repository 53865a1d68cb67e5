"""Control-variate form of the diag(Omega) estimator (test infrastructure only).

Not in the paper: an unbiased variance-reduction layer on top of Prop. 1.  Per
tree t and vertex v:
    X_t(v) = [the tree edge {u*, v} is present]       (Prop. 1: E[X] = Omega_vv)
    C_t(v) = [stack entry 0 of v selects u*]          (E[C] = p_v exactly)
where p_v is the exact discrete probability with which one stack entry selects
u* (slot 0 of the selector; 1/deg*(v) up to 2^-52).  A vertex whose first entry selects
u* can never lie on a popped cycle, so C = 1 implies X = 1.  For any
coefficient beta_v,
    Omega~_vv = mean_t X_t(v) - beta_v (mean_t C_t(v) - p_v)
is unbiased; the variance-optimal beta_v = (1 - Omega_vv) / (1 - p_v).  A
prediction g_v of Omega_vv gives beta_v = (1 - clip(g_v, p_v, 1)) / (1 - p_v).
"""
from __future__ import annotations

import numpy as np

from . import native


def p_root(g, alpha: float) -> np.ndarray:
    """Exact per-vertex probability that one stack entry selects u*."""
    d = g.degrees()
    if g.w is None:
        uniq, inv = np.unique(d, return_inverse=True)
        vals = np.array([native.p_root(int(x), alpha, 0.0, False) for x in uniq])
        return vals[inv]
    S = native.row_prefix(g)
    out = np.empty(g.n)
    for v in range(g.n):
        sd = S[g.rowptr[v + 1] - 1] if d[v] > 0 else 0.0
        out[v] = native.p_root(int(d[v]), alpha, float(sd), True)
    return out


def beta_from_prediction(gpred: np.ndarray, p: np.ndarray) -> np.ndarray:
    """beta_v = (1 - clip(g_v, p_v, 1)) / (1 - p_v); a prediction that is not a
    number is read as p_v (beta_v = 1), which keeps the estimator unbiased."""
    gpred = np.asarray(gpred, dtype=np.float64)
    gg = np.where(np.isnan(gpred), p, np.clip(gpred, p, 1.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(p < 1.0, (1.0 - gg) / (1.0 - p), 0.0)
    return b


def combine(R: np.ndarray, C: np.ndarray, tau: int, p: np.ndarray, beta: np.ndarray) -> np.ndarray:
    return R.astype(np.float64) / tau - beta * (C.astype(np.float64) / tau - p)
