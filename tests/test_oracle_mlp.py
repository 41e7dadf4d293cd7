"""Pins of the FP64 support-proposal network: central finite differences of
the loss for every parameter, GELU against its definition, Adam against a
hand-rolled first step."""
import math

import numpy as np
import pytest

from oracle import mlp


def small_net(seed=0, d=10, h=7, q=5, B=6):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, d))
    T = (rng.random((B, q)) < 0.3).astype(float)
    P = dict(W1=rng.standard_normal((h, d)) * 0.5, b1=rng.standard_normal(h) * 0.1,
             W2=rng.standard_normal((q, h)) * 0.5, b2=rng.standard_normal(q) * 0.1)
    return X, T, P


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2"])
def test_gradients_match_central_differences(name):
    X, T, P = small_net()
    _, g = mlp.loss_and_grads(X, T, **P)
    eps = 1e-6
    num = np.zeros_like(P[name])
    for idx in np.ndindex(P[name].shape):
        Pp = {k: v.copy() for k, v in P.items()}
        Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][idx] += eps
        Pm[name][idx] -= eps
        num[idx] = (mlp.loss_and_grads(X, T, **Pp)[0] - mlp.loss_and_grads(X, T, **Pm)[0]) / (2 * eps)
    rel = np.abs(num - g[name]).max() / np.abs(num).max()
    assert rel < 1e-6, rel


def test_gelu_definition_and_derivative():
    u = np.linspace(-4, 4, 81)
    Phi = np.array([0.5 * (1 + math.erf(x / math.sqrt(2))) for x in u])
    assert np.allclose(mlp.gelu(u), u * Phi, atol=1e-15)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(u), (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h), atol=1e-8)


def test_inputs_are_normalised_column_vec():
    Y = np.arange(2 * 3 * 4, dtype=float).reshape(2, 3, 4)
    X = mlp.inputs(Y)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0)
    assert np.allclose(X[1] * np.linalg.norm(Y[1]), Y[1].flatten(order="F"))
    assert np.all(mlp.inputs(np.zeros((1, 2, 2))) == 0)


def test_adam_first_step_is_signed_lr():
    p, g = np.array([1.0, -2.0, 3.0]), np.array([0.5, -0.1, 0.0])
    with np.errstate(invalid="ignore"):           # entry 3: 0 / 0 with eps = 0, not checked
        p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p1[:2], p[:2] - 0.01 * np.sign(g[:2]))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
