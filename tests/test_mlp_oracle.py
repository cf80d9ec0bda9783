"""Pins for the fp64 network oracle (oracle/mlp.py)."""
import numpy as np

from oracle import mlp


def rand_problem(seed, B=7, D=5, H=6):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=H * D + 2 * H + 1)
    X = rng.normal(size=(B, D))
    T = rng.normal(size=B)
    return p, X, T, D, H


def test_gradient_matches_central_finite_differences():
    p, X, T, D, H = rand_problem(1)
    L, g = mlp.loss_and_grad(p, X, T, D, H)
    eps = 1e-6
    for i in range(p.size):
        q = p.copy()
        q[i] += eps
        lp = mlp.loss_and_grad(q, X, T, D, H)[0]
        q[i] -= 2 * eps
        lm = mlp.loss_and_grad(q, X, T, D, H)[0]
        assert abs((lp - lm) / (2 * eps) - g[i]) < 1e-5 * max(1.0, abs(g[i])), i


def test_zero_first_layer_gives_constant_output():
    D, H = 3, 4
    p = np.zeros(H * D + 2 * H + 1)
    p[H * D: H * D + H] = [1.0, -1.0, 2.0, 0.5]     # b1
    p[H * D + H: H * D + 2 * H] = [1.0, 1.0, 1.0, 2.0]  # w2
    p[-1] = 0.25
    X = np.random.default_rng(0).normal(size=(5, D))
    # relu(b1) . w2 + b2 = 1 + 0 + 2 + 1 + 0.25
    assert np.allclose(mlp.forward(p, X, D, H), 4.25)


def test_single_active_unit_is_linear():
    D, H = 2, 1
    p = np.array([3.0, -2.0, 0.5, 4.0, 1.0])         # W1 = [3, -2], b1 = 0.5, w2 = 4, b2 = 1
    X = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    # z = 3.5, -1.5, 1.5 -> relu 3.5, 0, 1.5 -> y = 15, 1, 7
    assert np.allclose(mlp.forward(p, X, D, H), [15.0, 1.0, 7.0])
    L, g = mlp.loss_and_grad(p, X, np.array([15.0, 1.0, 6.0]), D, H)
    assert np.isclose(L, 1.0 / 3.0)                    # only the last sample is off, by 1
    # dL/db2 = 2 * 1 / 3; dL/dw2 = (2/3) * relu(z_3) = 1.0
    assert np.isclose(g[-1], 2.0 / 3.0) and np.isclose(g[3], 1.0)


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 0.0])
    g = np.array([0.3, -5.0, 0.0])
    q, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 0.1, 0.9, 0.999, 1e-12, 1)
    # with bias correction the first step is lr * g / |g|
    assert np.allclose(q, [0.9, -1.9, 0.0])
