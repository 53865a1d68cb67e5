"""Training and use of the learned control variate (not in the paper).

The network predicts g_v ~ Omega_vv; fc_forest_farness turns it into the
coefficient beta_v = (1 - g_v)/(1 - p_v) of the control variate C (first stack
entry of v selects u*), which keeps the estimator unbiased for any g.  Targets
are diag(Omega) estimates of the plain estimator on smaller graphs, produced by
the same sampler.  All arithmetic runs in libfc.so; this module only sequences
the calls (features, loss/gradient, Adam) and holds the parameter vector.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fc


def init_params(seed: int, device=None) -> torch.Tensor:
    """He-normal first layer, 1/sqrt(H) second layer, zero biases (seeded)."""
    count = fc.mlp_param_count()
    hid = (count - 1) // 6
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(count, dtype=np.float32)
    p[: hid * 4] = rng.normal(0.0, np.sqrt(2.0 / 4), size=hid * 4)
    p[hid * 5: hid * 6] = rng.normal(0.0, np.sqrt(1.0 / hid), size=hid)
    dev = device or torch.device("cuda", torch.cuda.current_device())
    return torch.from_numpy(p).to(dev)


def plain_targets(G: "fc.Graph", tau: int, seed: int, alpha_idx: int = 0) -> torch.Tensor:
    """diag(Omega) from tau trees of the plain estimator (Prop. 1), float32."""
    out = G.sample(seed, tau, with_C=False)
    diag, _, _ = G.farness(out["R"], tau, alpha_idx=alpha_idx)
    return diag.to(torch.float32)


def train(data, steps: int = 600, lr: float = 3e-3, seed: int = 0, params=None, log_every: int = 0):
    """Full-batch Adam over a list of (G, X, y, alpha_idx); the library averages
    the graphs' gradients (fc_mlp_loss_grad_acc with weight 1/#graphs).
    Returns (params, loss history)."""
    if params is None:
        params = init_params(seed)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    w = 1.0 / len(data)
    hist = []
    for step in range(1, steps + 1):
        for i, (G, X, y, a) in enumerate(data):
            G.mlp_loss_grad_acc(X, y, params, grad, loss, w, i > 0, alpha_idx=a)
        fc.mlp_adam(params, grad, m, v, step, lr)
        if log_every and step % log_every == 0:
            hist.append((step, float(loss.item())))
    return params, hist


def predict(G: "fc.Graph", params: torch.Tensor, alpha_idx: int = 0) -> torch.Tensor:
    X = G.features(alpha_idx)
    return G.mlp_forward(X, params, alpha_idx=alpha_idx)
