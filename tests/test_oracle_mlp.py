"""Pins of oracle.mlp: finite differences of the loss, closed forms."""

import math

import numpy as np

from oracle import mlp

rng = np.random.default_rng(3)


def small_problem(F=12, H=10, O=16, N=7):
    theta = rng.standard_normal(mlp.n_params(F, H, O)) * 0.3
    X = rng.standard_normal((N, F))
    lens = rng.choice([2, 4, 8, 16], size=N)
    T = np.abs(rng.standard_normal((N, O))) * (np.arange(O)[None, :] < lens[:, None])
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    return theta, X, T, lens


def test_gradient_matches_central_differences():
    F, H, O = 12, 10, 16
    theta, X, T, lens = small_problem(F, H, O)
    L, g = mlp.loss_and_grad(theta, X, T, lens, F, H, O)
    idx = rng.choice(theta.size, size=60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        fd = (mlp.loss(tp, X, T, lens, F, H, O) - mlp.loss(tm, X, T, lens, F, H, O)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    # GELU(x) -> x for large x and -> 0 for very negative x.
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    # Equal logits give the uniform message (Remark 2's initial message).
    u, _ = mlp.message_from_logits(np.zeros((1, 16)), [16])
    np.testing.assert_allclose(u, np.full((1, 16), 0.25))
    # A message equal to its target has zero loss.
    o = rng.standard_normal((3, 16))
    u, _ = mlp.message_from_logits(o, [4, 8, 16])
    c = np.sum(u * u, axis=1)
    assert np.allclose(1 - c * c, 0.0)


def test_adam_first_step_moves_by_lr():
    theta = np.zeros(5)
    g = np.array([1.0, -2.0, 3.0, 0.5, -0.1])
    m, v = np.zeros(5), np.zeros(5)
    mlp.adam(theta, g, m, v, 1, lr=1e-2)
    np.testing.assert_allclose(theta, -1e-2 * np.sign(g), rtol=1e-6)
