"""Pins for the reference MLP: finite-difference gradients and one Adam step."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(3) + 0.05 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((17, 8))
    T = rng.standard_normal((17, 2))
    L, g = mlp.loss_grad(theta, X, T, lam=3.0)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM); e[i] = h
        fd = (mlp.loss_grad(theta + e, X, T, 3.0)[0] - mlp.loss_grad(theta - e, X, T, 3.0)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd)), i


def test_loss_is_asymmetric():
    theta = mlp.init_params(0)
    X = np.zeros((1, 8))
    Y, _ = mlp.forward(theta, X)
    over = mlp.loss_grad(theta, X, Y - 0.5, lam=4.0)[0]
    under = mlp.loss_grad(theta, X, Y + 0.5, lam=4.0)[0]
    assert abs(under / over - 5.0) < 1e-12


def test_adam_first_step_is_signed_lr():
    theta = np.zeros(4)
    g = np.array([1.0, -2.0, 0.5, 0.0])
    t2, m, v = mlp.adam_step(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    # first bias-corrected step: -lr * g / (|g| + eps)
    assert np.allclose(t2, -0.1 * g / (np.abs(g) + 1e-8))
