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


def test_adam_second_and_third_steps_follow_the_bias_correction():
    # Hand derivation (Kingma & Ba, Algorithm 1): with zero gradients before
    # step t and gradient g at step t, the moments are m = (1-b1) g and
    # v = (1-b2) g^2, so the corrected moments are g / (1 + b1 + ... + b1^(t-1))
    # and g^2 / (1 + b2 + ... + b2^(t-1)) and the step is
    #   lr sign(g) sqrt(1 + b2 + ... + b2^(t-1)) / (1 + b1 + ... + b1^(t-1)).
    # With b1 = 0.9, b2 = 0.999: t = 2 gives sqrt(1.999) / 1.9 = 0.7441368...,
    # t = 3 gives sqrt(2.997001) / 2.71 = 0.6388136...  A correction by
    # beta**1 at every step would give 1.0 and 0.964...; no correction 3.16.
    lr, b1, b2 = 0.1, 0.9, 0.999
    for t, expect in ((2, 0.7441368), (3, 0.6388136)):
        p = np.array([1.0, 1.0])
        m = np.zeros(2)
        v = np.zeros(2)
        for step in range(1, t + 1):
            g = np.array([0.25, -4.0]) if step == t else np.zeros(2)
            p, m, v = mlp.adam_step(p, g, m, v, lr, b1, b2, 0.0 if step == t else 1.0, step)
        assert np.allclose(p, [1.0 - lr * expect, 1.0 + lr * expect], rtol=0, atol=1e-7), (t, p)


def test_adam_two_steps_with_nonzero_history():
    # b1 = b2 = 0.5, lr = 1, eps = 0, g1 = 2 then g2 = 4 (worked by hand):
    # step 1: m = 1, v = 2, corrected 2 and 4, step 2 / 2 = 1     -> p = -1
    # step 2: m = 0.5 + 2 = 2.5, v = 1 + 8 = 9; corrections 1 - 0.25 = 0.75
    # for both: m^ = 10/3, v^ = 12, step (10/3) / sqrt(12) = 0.9622504 -> p = -1.9622504
    p, m, v = mlp.adam_step(np.array([0.0]), np.array([2.0]), np.zeros(1), np.zeros(1), 1.0, 0.5, 0.5, 0.0, 1)
    assert np.allclose(p, [-1.0]) and np.allclose(m, [1.0]) and np.allclose(v, [2.0])
    p, m, v = mlp.adam_step(p, np.array([4.0]), m, v, 1.0, 0.5, 0.5, 0.0, 2)
    assert np.allclose(m, [2.5]) and np.allclose(v, [9.0])
    assert np.allclose(p, [-1.9622504], rtol=0, atol=1e-7)
