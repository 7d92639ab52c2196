"""Float64 reference of the learned warm start for out-of-sample embedding.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline arm, never by the library.

The paper has no learned component; this network is the "learned part" added beside the
method: it maps a new object's dissimilarities to a fixed set of in-sample landmarks to a
starting position for the out-of-sample Guttman iterations (Sec. 3), which then refine
it.  Definitions written out plainly:

* features: for landmarks l_1..l_L (in-sample indices shared by all modalities) and a
  per-modality normaliser c_j (the mean of Delta_j), the input is the m*L vector
  [delta_j(l_t) / c_j], modality-major, rounded to float16 by the library;
* network: h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), yhat = W3 h2 + b3, with
  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2;
* target: the commensurate position ybar = mean_j y_j of the method's own out-of-sample
  solution; the warm start puts every y_j(0) = yhat;
* loss: L = 1/(2B) sum_b ||yhat_b - ybar_b||^2 over a batch of B objects;
* optimiser: Adam (Kingma & Ba 2015) with bias correction.

Parameters are one flat float vector: W1 (H x I), b1 (H), W2 (H x H), b2 (H), W3 (O x H),
b3 (O), each matrix row-major (row = output unit).
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def param_count(n_in: int, hidden: int, n_out: int) -> int:
    return hidden * n_in + hidden + hidden * hidden + hidden + n_out * hidden + n_out


def unpack(theta: np.ndarray, n_in: int, hidden: int, n_out: int):
    """Views (W1, b1, W2, b2, W3, b3) into the flat parameter vector."""
    theta = np.asarray(theta, dtype=np.float64)
    shapes = [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (n_out, hidden), (n_out,)]
    out, off = [], 0
    for shp in shapes:
        size = int(np.prod(shp))
        out.append(theta[off:off + size].reshape(shp))
        off += size
    assert off == theta.size
    return out


def gelu(z: np.ndarray) -> np.ndarray:
    """z * Phi(z) with the standard normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2."""
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d/dz [z Phi(z)] = Phi(z) + z phi(z), phi the standard normal density."""
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(theta: np.ndarray, X: np.ndarray, n_in: int, hidden: int, n_out: int):
    """Network output for the rows of X (B x n_in) and the pre-activations."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden, n_out)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, Y, n_in, hidden, n_out) -> float:
    yhat, _ = forward(theta, X, n_in, hidden, n_out)
    r = yhat - np.asarray(Y, dtype=np.float64)
    return float(0.5 * np.sum(r * r) / X.shape[0])


def gradient(theta, X, Y, n_in, hidden, n_out) -> Tuple[float, np.ndarray]:
    """Loss and its gradient by the chain rule, layer by layer from the output."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden, n_out)
    yhat, (X, z1, h1, z2, h2) = forward(theta, X, n_in, hidden, n_out)
    B = X.shape[0]
    r = yhat - np.asarray(Y, dtype=np.float64)
    L = float(0.5 * np.sum(r * r) / B)
    dy = r / B                                  # dL/dyhat
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(theta, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step t >= 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def features(delta_new: np.ndarray, landmarks: np.ndarray, inv_mean: np.ndarray) -> np.ndarray:
    """Network inputs for new objects: delta_new (k, m, n) -> (k, m*L), entry
    [o, j*L + t] = delta_new[o, j, landmarks[t]] * inv_mean[j] (before float16 rounding)."""
    delta_new = np.asarray(delta_new, dtype=np.float64)
    k, m, _ = delta_new.shape
    L = len(landmarks)
    out = np.empty((k, m * L))
    for j in range(m):
        out[:, j * L:(j + 1) * L] = delta_new[:, j, :][:, landmarks] * inv_mean[j]
    return out
