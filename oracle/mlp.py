"""FP64 reference of the learned control-variate network (test infrastructure only).

Not in the paper.  A two-layer perceptron predicts g_v ~ Omega_vv from local
features of v; the prediction only sets the control-variate coefficient
beta_v = (1 - g_v) / (1 - p_v), so the estimator stays unbiased whatever the
network outputs.

Features of v (alpha > 0):
    x0 = log(1 + deg(v))                      degree
    x1 = log(1 + alpha * d_w(v))              weighted degree in G* minus the u*-edge
    x2 = log(1 + sum_{u in N(v)} deg(u))      2-hop degree sum
    x3 = log(alpha)
Network: h = relu(W1 x + b1) (W1: H x 4), z = w2 . h + b2,
         g = p + (1 - p) sigmoid(z)   (so g in (p_v, 1) and beta = 1 - sigmoid(z)).
Loss:    mean over vertices of (g - y)^2 for targets y.
Optimiser: Adam (Kingma & Ba, ICLR 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128
N_FEAT = 4


def features(g, alpha: float) -> np.ndarray:
    d = g.degrees().astype(np.float64)
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    dw = np.bincount(src, weights=w, minlength=g.n)
    s2 = np.bincount(src, weights=d[g.colidx], minlength=g.n)
    X = np.empty((g.n, N_FEAT))
    X[:, 0] = np.log1p(d)
    X[:, 1] = np.log1p(alpha * dw)
    X[:, 2] = np.log1p(s2)
    X[:, 3] = np.log(alpha)
    return X


def init_params(seed: int, hidden: int = HIDDEN) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    return {
        "W1": rng.normal(0.0, np.sqrt(2.0 / N_FEAT), size=(hidden, N_FEAT)),
        "b1": np.zeros(hidden),
        "w2": rng.normal(0.0, np.sqrt(1.0 / hidden), size=hidden),
        "b2": np.zeros(1),
    }


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params: dict, X: np.ndarray, p: np.ndarray):
    pre = X @ params["W1"].T + params["b1"]
    h = np.maximum(pre, 0.0)
    z = h @ params["w2"] + params["b2"][0]
    s = _sigmoid(z)
    g = p + (1.0 - p) * s
    return g, {"pre": pre, "h": h, "z": z, "s": s}


def loss_and_grads(params: dict, X: np.ndarray, p: np.ndarray, y: np.ndarray):
    g, c = forward(params, X, p)
    N = X.shape[0]
    r = g - y
    loss = float(np.mean(r * r))
    dg = 2.0 * r / N
    dz = dg * (1.0 - p) * c["s"] * (1.0 - c["s"])
    grads = {
        "w2": c["h"].T @ dz,
        "b2": np.array([dz.sum()]),
    }
    dh = np.outer(dz, params["w2"])
    dpre = dh * (c["pre"] > 0)
    grads["W1"] = dpre.T @ X
    grads["b1"] = dpre.sum(axis=0)
    return loss, grads


def adam_step(params: dict, grads: dict, state: dict, lr: float, t: int,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """In-place Adam update; ``t`` is the 1-based step number."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m *= b1
        m += (1.0 - b1) * grads[k]
        v *= b2
        v += (1.0 - b2) * grads[k] ** 2
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        params[k] -= lr * mh / (np.sqrt(vh) + eps)
