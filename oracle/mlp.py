"""FP64 reference of the sub-cycle-count predictor.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).  The
predictor is not part of the paper; it only reorders work, the criterion of
Sec. IV still decides every sub-step.  Plain numpy, float64, no batching tricks.

Network: 6 -> 64 -> 64 -> 8, ReLU on the two hidden layers, softmax
cross-entropy over the 8 classes k = 0..7 (4^k sub-steps, Algorithm 1).
Row-vector convention: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2),
z = h2 W3^T + b3, W_l of shape (out, in).

Features of one particle (local field, momentum, gamma):
  phi = (asinh|E_y|, asinh|B_z|, asinh p_x, asinh p_y, asinh p_z, log gamma).

Pins (tests/test_oracle_mlp.py): central finite differences of the loss for
every parameter tensor; the closed forms d(loss)/dz = (softmax(z) - onehot)/N
and loss = log 8 for zero logits.
"""
from __future__ import annotations

import numpy as np

SIZES = (6, 64, 64, 8)


def features(ey, bz, px, py, pz):
    ey, bz, px, py, pz = (np.asarray(a, dtype=np.float64) for a in (ey, bz, px, py, pz))
    g = np.sqrt(1.0 + px * px + py * py + pz * pz)
    return np.stack([np.arcsinh(np.abs(ey)), np.arcsinh(np.abs(bz)), np.arcsinh(px),
                     np.arcsinh(py), np.arcsinh(pz), np.log(g)], axis=1)


def init_params(seed: int = 0):
    """He-uniform weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = {}
    for l, (fi, fo) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        bound = np.sqrt(6.0 / fi)
        params[f"W{l}"] = rng.uniform(-bound, bound, size=(fo, fi))
        params[f"b{l}"] = np.zeros(fo)
    return params


def forward(params, X):
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ params["W1"].T + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ params["W3"].T + params["b3"]
    return z, (X, a1, h1, a2, h2)


def loss_and_grads(params, X, y):
    """Mean softmax cross-entropy over the batch and its gradients."""
    z, (X, a1, h1, a2, h2) = forward(params, X)
    y = np.asarray(y, dtype=np.int64)
    N = X.shape[0]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    s = e.sum(axis=1, keepdims=True)
    logp = (z - zmax) - np.log(s)
    loss = -logp[np.arange(N), y].mean()
    dz = e / s
    dz[np.arange(N), y] -= 1.0
    dz /= N
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = dz @ params["W3"]
    da2 = dh2 * (a2 > 0.0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ params["W2"]
    da1 = dh1 * (a1 > 0.0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return loss, g


def predict(params, X):
    z, _ = forward(params, X)
    return np.argmax(z, axis=1)
