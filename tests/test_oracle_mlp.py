"""Pins of the oracle's warm-start network (FP64): GELU values, identity layer, finite differences."""
import numpy as np

from oracle import mlp


def test_gelu_special_values():
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15      # Phi(1)
    assert abs(mlp.gelu(np.array(-1.0)) + 0.15865525393145707) < 1e-15    # -(1 - Phi(1))
    assert abs(mlp.gelu(np.array(12.0)) - 12.0) < 1e-12 and abs(mlp.gelu(np.array(-12.0))) < 1e-12
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(z)).max() < 1e-8


def test_single_identity_layer_is_affine():
    rng = np.random.default_rng(0)
    W, b, X = rng.normal(size=(3, 5)), rng.normal(size=3), rng.normal(size=(7, 5))
    Y, _ = mlp.forward([(W, b)], X)
    assert np.abs(Y - (X @ W.T + b)).max() < 1e-14


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    dims = [4, 9, 7, 6]
    params = [(rng.normal(size=(dims[i + 1], dims[i])) * 0.5, rng.normal(size=dims[i + 1]) * 0.1)
              for i in range(3)]
    X, T = rng.normal(size=(11, 4)), rng.normal(size=(11, 6))
    Y, cache = mlp.forward(params, X)
    L, dY = mlp.mse(Y, T)
    grads = mlp.backward(params, cache, dY)
    h = 1e-6
    for li in range(3):
        for idx in [(0, 0), (dims[li + 1] - 1, dims[li] - 1), (1, 2)]:
            W, b = params[li]
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params)
            pp[li] = (Wp, b)
            Lp = mlp.mse(mlp.forward(pp, X)[0], T)[0]
            pp[li] = (Wm, b)
            Lm = mlp.mse(mlp.forward(pp, X)[0], T)[0]
            assert abs((Lp - Lm) / (2 * h) - grads[li][0][idx]) < 1e-7
        bp = params[li][1].copy()
        bp[0] += h
        pp = list(params)
        pp[li] = (params[li][0], bp)
        Lp = mlp.mse(mlp.forward(pp, X)[0], T)[0]
        assert abs((Lp - L) / h - grads[li][1][0]) < 1e-5
