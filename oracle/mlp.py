"""FP64 CPU oracle of the per-element MLP of the learned preconditioner.

TEST INFRASTRUCTURE ONLY: used by the tests (gradient checks of the GPU
training kernels), never by the product path.  Shares no code with the CUDA
library.

Network (per element, no weight sharing across layers):
    Z1 = X W1^T + b1,  H1 = gelu(Z1)
    Z2 = H1 W2^T + b2, H2 = gelu(Z2)
    Y  = H2 W3^T + b3                      (linear output)
with gelu(z) = z Phi(z), Phi the standard normal CDF, written with erf:
    gelu(z) = 0.5 z (1 + erf(z / sqrt 2)),  gelu'(z) = Phi(z) + z phi(z).
Loss: L = 0.5 * mean over samples and outputs of (Y - T)^2.
Backward by the chain rule, plain numpy matmuls (library primitive).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT2PI * np.exp(-0.5 * z * z)


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss(params, X, T):
    Y, _ = forward(params, X)
    return 0.5 * np.mean((Y - T) ** 2)


def grads(params, X, T):
    """(loss, [dW1, db1, dW2, db2, dW3, db3])."""
    W1, b1, W2, b2, W3, b3 = params
    Y, (X, Z1, H1, Z2, H2) = forward(params, X)
    M, O = Y.shape
    L = 0.5 * np.mean((Y - T) ** 2)
    dY = (Y - T) / (M * O)
    dW3 = dY.T @ H2
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3) * gelu_grad(Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return L, [dW1, db1, dW2, db2, dW3, db3]


def init(in_dim, hidden, out_dim, seed=0):
    """Plain float64 initialisation for the oracle's own tests."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, in_dim)) / math.sqrt(in_dim)
    W2 = rng.standard_normal((hidden, hidden)) / math.sqrt(hidden)
    W3 = rng.standard_normal((out_dim, hidden)) / math.sqrt(hidden)
    return [W1, 0.1 * rng.standard_normal(hidden), W2, 0.1 * rng.standard_normal(hidden), W3,
            0.1 * rng.standard_normal(out_dim)]
