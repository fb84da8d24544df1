"""FP64 reference of the error-estimator network: forward, backward and Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper monitors the reconstruction error by computing it (Eq. 2.20).  The
estimator that predicts it from reduced quantities is not in the paper; this
module restates only textbook pieces so that the GPU kernels can be checked:

* a two-hidden-layer perceptron with tanh activations,
      h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = w3 . h2 + b3;
* the mean-squared-error loss L = mean_i (y_i - t_i)^2;
* back-propagation of L;
* Adam (Kingma and Ba, 2015) with bias correction.

Parameters live in one flat vector in the order W1 (H x F, row-major), b1 (H),
W2 (H x H, row-major), b2 (H), w3 (H), b3 (1).
"""

from __future__ import annotations

import numpy as np

__all__ = ["n_params", "unpack", "forward", "loss_and_grad", "adam_update", "init_params"]


def n_params(F: int, H: int) -> int:
    return H * F + H + H * H + H + H + 1


def unpack(theta: np.ndarray, F: int, H: int):
    o = 0
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta: np.ndarray, X: np.ndarray, F: int, H: int) -> np.ndarray:
    """y for every row of X (B x F)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, F, H)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, F: int, H: int):
    """(L, dL/dtheta) for L = mean (y - t)^2, by the chain rule."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, F, H)
    B = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    y = h2 @ w3 + b3
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B                       # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = np.sum(dy)
    dh2 = np.outer(dy, w3)
    da2 = dh2 * (1.0 - h2 * h2)
    g_W2 = da2.T @ h1
    g_b2 = np.sum(da2, axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (1.0 - h1 * h1)
    g_W1 = da1.T @ X
    g_b1 = np.sum(da1, axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return L, g


def adam_update(theta, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                eps: float = 1e-8):
    """One Adam step (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def init_params(F: int, H: int, rng: np.random.Generator) -> np.ndarray:
    """Glorot-uniform weights, zero biases."""
    def glorot(fan_out, fan_in):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_out, fan_in))
    return np.concatenate([glorot(H, F).ravel(), np.zeros(H), glorot(H, H).ravel(), np.zeros(H),
                           glorot(1, H).ravel(), [0.0]])
