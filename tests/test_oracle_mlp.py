"""Pins of the FP64 predictor oracle (oracle/mlp.py) against finite differences
and closed forms of softmax cross-entropy."""
from __future__ import annotations

import numpy as np

from oracle import mlp


def _batch(n=37, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 6))
    y = rng.integers(0, 8, n)
    return X, y


def test_gradients_match_central_differences():
    P = mlp.init_params(3)
    for k in P:                     # non-zero biases so every term is exercised
        if k.startswith("b"):
            P[k] = np.random.default_rng(7).standard_normal(P[k].shape) * 0.1
    X, y = _batch()
    _, g = mlp.loss_and_grads(P, X, y)
    rng = np.random.default_rng(11)
    eps = 1e-6
    for name, W in P.items():
        flat = W.reshape(-1)
        for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = mlp.loss_and_grads(P, X, y)
            flat[idx] = old - eps
            lm, _ = mlp.loss_and_grads(P, X, y)
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            got = g[name].reshape(-1)[idx]
            assert abs(num - got) <= 1e-6 * max(1.0, abs(num)), (name, idx, num, got)


def test_zero_network_closed_forms():
    P = {k: np.zeros_like(v) for k, v in mlp.init_params(0).items()}
    X, y = _batch(16)
    loss, g = mlp.loss_and_grads(P, X, y)
    assert abs(loss - np.log(8.0)) < 1e-15
    # d loss / d b3 = mean(softmax - onehot) = 1/8 - frequency of each class
    freq = np.bincount(y, minlength=8) / len(y)
    np.testing.assert_allclose(g["b3"], 1.0 / 8 - freq, atol=1e-15)
    assert not np.any(g["W1"]) and not np.any(g["W2"])


def test_features_hand_computed():
    """phi = (asinh|E_y|, asinh|B_z|, asinh p_x, asinh p_y, asinh p_z, log gamma)
    at E_y = 3, B_z = -4, p = (0, 1, -2), against values worked out by hand from
    asinh u = ln(u + sqrt(u^2 + 1)) and gamma = sqrt(1 + 0 + 1 + 4) = sqrt 6:
    ln(3 + sqrt 10), ln(4 + sqrt 17), 0, ln(1 + sqrt 2), -ln(2 + sqrt 5), ln 6 / 2."""
    f = mlp.features([3.0], [-4.0], [0.0], [1.0], [-2.0])
    want = [1.8184464592320668, 2.0947125472611012, 0.0, 0.8813735870195430,
            -1.4436354751788103, 0.8958797346140275]
    np.testing.assert_allclose(f[0], want, rtol=1e-15, atol=0)
