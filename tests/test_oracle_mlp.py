"""Pins for the MLP oracle: GELU against scipy's normal CDF (z Phi(z)) and
its derivative against finite differences; the backward pass against
central finite differences of the loss for every parameter tensor."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_is_z_times_normal_cdf():
    z = np.linspace(-8, 8, 2001)
    np.testing.assert_allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)
    assert mlp.gelu(0.0) == 0.0


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(100 + seed)
    I, H, O, M = 7, 6, 5, 4
    params = mlp.init(I, H, O, seed)
    X = rng.standard_normal((M, I))
    T = rng.standard_normal((M, O))
    L, g = mlp.grads(params, X, T)
    assert abs(L - mlp.loss(params, X, T)) < 1e-15
    h = 1e-6
    for p, gp in zip(params, g):
        flat = p.reshape(-1)
        gflat = gp.reshape(-1)
        for q in range(flat.size):
            old = flat[q]
            flat[q] = old + h
            lp = mlp.loss(params, X, T)
            flat[q] = old - h
            lm = mlp.loss(params, X, T)
            flat[q] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[q]) <= 1e-7 * max(1.0, abs(fd)), (q, fd, gflat[q])


def test_planted_mistake_in_backward_is_caught():
    # a transposed weight in the second layer's backward must break the FD check
    rng = np.random.default_rng(7)
    I, H, O, M = 5, 5, 5, 3
    params = mlp.init(I, H, O, 3)
    X, T = rng.standard_normal((M, I)), rng.standard_normal((M, O))
    W1, b1, W2, b2, W3, b3 = params
    Y, (X_, Z1, H1, Z2, H2) = mlp.forward(params, X)
    dY = (Y - T) / Y.size
    dZ2 = (dY @ W3) * mlp.gelu_grad(Z2)
    wrong_dZ1 = (dZ2 @ W2.T) * mlp.gelu_grad(Z1)  # planted: W2 transposed
    wrong_dW1 = wrong_dZ1.T @ X
    _, g = mlp.grads(params, X, T)
    assert np.max(np.abs(wrong_dW1 - g[0])) > 1e-6
