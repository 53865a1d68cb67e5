"""FP64 conjugate-gradient ground truth on I + alpha L (test infrastructure only).

The paper takes its ground truth Omega[v, v] from a CG solver at tolerance 1e-9
(Sec. 6.1, the accuracy measurement) and checks it against NumPy's pinv.
This module is the same idea written out plainly: textbook CG (Hestenes-Stiefel)
on the SPD matrix A = I + alpha L with scipy's sparse product as the only
library step; column e_v of the solution gives Omega[:, v] and its v-th entry
Omega[v, v].  Several right-hand sides run as independent CG recurrences side by
side (no block coupling).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def system_matrix(g, alpha: float) -> sp.csr_matrix:
    """A = I + alpha L as a scipy CSR matrix in FP64."""
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    Adj = sp.csr_matrix((w, g.colidx.astype(np.int64), g.rowptr), shape=(g.n, g.n))
    dw = np.asarray(Adj.sum(axis=1)).ravel()
    return (sp.diags(1.0 + alpha * dw) - alpha * Adj).tocsr()


def cg(A: sp.csr_matrix, B: np.ndarray, rel_tol: float = 1e-12, max_iter: int = 10_000):
    """Independent CG for each column of B (n x k).  Returns (X, iterations)."""
    B = np.asarray(B, dtype=np.float64)
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None]
    X = np.zeros_like(B)
    Rr = B.copy()
    P = Rr.copy()
    rs = np.einsum("ij,ij->j", Rr, Rr)
    bnorm = np.sqrt(np.einsum("ij,ij->j", B, B))
    bnorm[bnorm == 0] = 1.0
    it = 0
    active = np.sqrt(rs) > rel_tol * bnorm
    while active.any() and it < max_iter:
        AP = A @ P
        pAp = np.einsum("ij,ij->j", P, AP)
        a = np.where(active, rs / np.where(pAp == 0, 1.0, pAp), 0.0)
        X += P * a
        Rr -= AP * a
        rs_new = np.einsum("ij,ij->j", Rr, Rr)
        b = np.where(active, rs_new / np.where(rs == 0, 1.0, rs), 0.0)
        P = Rr + P * b
        rs = rs_new
        active = np.sqrt(rs) > rel_tol * bnorm
        it += 1
    return (X[:, 0] if squeeze else X), it


def omega_columns(g, alpha: float, vertices, rel_tol: float = 1e-12):
    """Omega[:, v] for each v in ``vertices`` (n x k) by CG on I + alpha L."""
    vertices = np.asarray(vertices, dtype=np.int64)
    B = np.zeros((g.n, vertices.size))
    B[vertices, np.arange(vertices.size)] = 1.0
    X, _ = cg(system_matrix(g, alpha), B, rel_tol=rel_tol)
    return X


def omega_diag_at(g, alpha: float, vertices, rel_tol: float = 1e-12) -> np.ndarray:
    vertices = np.asarray(vertices, dtype=np.int64)
    X = omega_columns(g, alpha, vertices, rel_tol)
    return X[vertices, np.arange(vertices.size)]
