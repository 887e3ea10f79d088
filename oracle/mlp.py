"""Oracle: the warm-start network in FP64 (test infrastructure only).

Not part of the paper: a fully connected network z_l = W_l y_{l-1} + b_l, y_l = GELU(z_l) on hidden
layers (GELU(z) = z Phi(z) = z (1 + erf(z/sqrt 2))/2), identity on the last layer, trained by mean
squared error.  forward/backward restate the chain rule layer by layer in FP64; the weights passed in
are whatever the device uses (BF16 values), so the comparison isolates the arithmetic.

Pins (tests/test_oracle_mlp.py): GELU special values, the identity layer as a plain product, and
the backward pass against central finite differences of the loss.
"""
from __future__ import annotations

from math import erf, sqrt

import numpy as np

_erf = np.vectorize(erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / sqrt(2.0)))


def gelu_grad(z):
    Phi = 0.5 * (1.0 + _erf(z / sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / sqrt(2.0 * np.pi)
    return Phi + z * phi


def forward(params, X):
    """params: list of (W [out, in], b [out]); returns (Y, cache) with cache = [(y_in, z)] per layer."""
    y = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(params):
        z = y @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        cache.append((y, z))
        y = gelu(z) if li < len(params) - 1 else z
    return y, cache


def mse(Y, T):
    d = Y - T
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, cache, dY):
    """Gradients [(dW, db)] of a scalar loss with dL/dY = dY."""
    grads = [None] * len(params)
    g = dY
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        y_in, z = cache[li]
        dz = g * gelu_grad(z) if li < len(params) - 1 else g
        grads[li] = (dz.T @ y_in, dz.sum(axis=0))
        g = dz @ np.asarray(W, np.float64)
    return grads
