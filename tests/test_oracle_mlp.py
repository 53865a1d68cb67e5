"""Pins of the oracle's FP64 control-variate network (forward/backward/Adam)."""
import numpy as np

import synth
from oracle import mlp


def _setup(seed=3):
    g = synth.barabasi_albert(120, 3, seed)
    X = mlp.features(g, 1.0)
    p = 1.0 / (1.0 + g.degrees())
    rng = np.random.default_rng(seed)
    y = np.clip(p + rng.random(g.n) * 0.2, 0, 1)
    return g, X, p, y


def test_gradients_match_central_differences():
    """Backward pass == FP64 central finite differences of the loss."""
    g, X, p, y = _setup()
    params = mlp.init_params(7, hidden=16)
    params["b1"] += 0.05
    _, grads = mlp.loss_and_grads(params, X, p, y)
    h = 1e-6
    for k in params:
        flat = params[k].ravel()
        for idx in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(params, X, p, y)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(params, X, p, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = grads[k].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_prediction_range_and_beta():
    """g = p + (1-p) sigmoid(z) lies in (p, 1], so beta = (1-g)/(1-p) in [0, 1)."""
    g, X, p, y = _setup()
    params = mlp.init_params(1)
    gp, c = mlp.forward(params, X, p)
    assert np.all(gp >= p) and np.all(gp <= 1)
    np.testing.assert_allclose((1 - gp) / (1 - p), 1 - c["s"], atol=1e-12)


def test_features_closed_form_star():
    """Star S_5 (centre 0): degrees 4/1, 2-hop sums 4 (centre) and 4 (leaves)."""
    g = synth.star(5)
    X = mlp.features(g, 2.0)
    np.testing.assert_allclose(X[0], [np.log(5), np.log(9), np.log(5), np.log(2)])
    np.testing.assert_allclose(X[1], [np.log(2), np.log(3), np.log(5), np.log(2)])


def test_adam_first_step_is_signed_lr():
    """At t = 1 the bias-corrected moments are g and g^2, so each parameter moves
    by -lr g / (|g| + eps)."""
    params = {"a": np.array([1.0, -2.0, 0.5])}
    grads = {"a": np.array([0.3, -4.0, 0.0])}
    st = {}
    mlp.adam_step(params, grads, st, lr=0.01, t=1)
    exp = np.array([1.0, -2.0, 0.5]) - 0.01 * grads["a"] / (np.abs(grads["a"]) + 1e-8)
    np.testing.assert_allclose(params["a"], exp, rtol=1e-12)


def test_training_reduces_loss():
    g, X, p, y = _setup(5)
    params = mlp.init_params(2, hidden=32)
    st = {}
    l0, _ = mlp.loss_and_grads(params, X, p, y)
    for t in range(1, 200):
        _, gr = mlp.loss_and_grads(params, X, p, y)
        mlp.adam_step(params, gr, st, lr=3e-3, t=t)
    l1, _ = mlp.loss_and_grads(params, X, p, y)
    assert l1 < 0.5 * l0
