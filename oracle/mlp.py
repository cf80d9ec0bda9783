"""fp64 reference of the plan cost-model network (test infrastructure only).

y = w2 . relu(W1 x + b1) + b2, loss L = (1/B) sum (y - t)^2, gradients by
the chain rule written out term by term; Adam as defined by Kingma & Ba
("Adam: a method for stochastic optimization", ICLR 2015, Algorithm 1).
Parameter layout: W1 [H x D] row-major, b1 [H], w2 [H], b2 [1].

Pinned in tests/test_mlp_oracle.py by central finite differences, closed
forms (zero weights, a single active unit) and hand-computed Adam steps 1-3.
"""
from __future__ import annotations

import numpy as np


def unpack(p: np.ndarray, D: int, H: int):
    p = np.asarray(p, dtype=np.float64)
    W1 = p[: H * D].reshape(H, D)
    b1 = p[H * D: H * D + H]
    w2 = p[H * D + H: H * D + 2 * H]
    b2 = p[H * D + 2 * H]
    return W1, b1, w2, b2


def forward(p, X, D, H):
    W1, b1, w2, b2 = unpack(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    Z = X @ W1.T + b1            # [B, H]
    A = np.maximum(Z, 0.0)
    return A @ w2 + b2


def loss_and_grad(p, X, T, D, H):
    W1, b1, w2, b2 = unpack(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    Z = X @ W1.T + b1
    A = np.maximum(Z, 0.0)
    Y = A @ w2 + b2
    R = Y - T
    L = float(np.sum(R * R) / B)
    dY = 2.0 * R / B                       # dL/dy_s
    g_b2 = np.sum(dY)
    g_w2 = A.T @ dY                        # sum_s dy_s a_s
    dZ = (dY[:, None] * w2[None, :]) * (Z > 0)
    g_b1 = dZ.sum(axis=0)
    g_W1 = dZ.T @ X
    g = np.concatenate([g_W1.ravel(), g_b1, g_w2, [g_b2]])
    return L, g


def adam_step(p, g, m, v, lr, beta1, beta2, eps, step):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
