"""FP64 reference of the support-proposal network (TEST INFRASTRUCTURE ONLY,
see the package docstring).

Input x = vec(Y) / ||Y||_F (column-order vec, Sec. I; 0 for a zero signal),
hidden h = GELU(W1 x + b1) with GELU(u) = u Phi(u) = 0.5 u (1 + erf(u/sqrt 2)),
scores z = W2 h + b2, one per atom pair q = i + n1*j.  Training target: the
multi-hot indicator of the 2D-OMP support; loss = mean over the batch of the
summed binary cross-entropy with logits, softplus(z) - t z.  Gradients are
the hand-derived backward pass; Adam is the standard bias-corrected update.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["inputs", "targets", "gelu", "gelu_grad", "forward", "loss_and_grads", "adam_step"]

_erf = np.vectorize(math.erf)


def inputs(Y) -> np.ndarray:
    Y = np.asarray(Y, dtype=np.float64)
    X = Y.transpose(0, 2, 1).reshape(Y.shape[0], -1)        # column-order vec
    nrm = np.linalg.norm(X, axis=1, keepdims=True)
    return np.where(nrm > 0, X / np.where(nrm > 0, nrm, 1.0), 0.0)


def targets(support, nq: int) -> np.ndarray:
    T = np.zeros((support.shape[0], nq))
    for b in range(support.shape[0]):
        for q in support[b]:
            if 0 <= q < nq:
                T[b, q] = 1.0
    return T


def gelu(u):
    return 0.5 * u * (1.0 + _erf(u / math.sqrt(2.0)))


def gelu_grad(u):
    return 0.5 * (1.0 + _erf(u / math.sqrt(2.0))) + u * np.exp(-0.5 * u * u) / math.sqrt(2 * math.pi)


def forward(X, W1, b1, W2, b2):
    pre = X @ W1.T + b1
    H = gelu(pre)
    return pre, H, H @ W2.T + b2


def _softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def loss_and_grads(X, T, W1, b1, W2, b2):
    B = X.shape[0]
    pre, H, Z = forward(X, W1, b1, W2, b2)
    loss = float(np.sum(_softplus(Z) - T * Z) / B)
    dZ = (1.0 / (1.0 + np.exp(-Z)) - T) / B
    gW2 = dZ.T @ H
    gb2 = dZ.sum(axis=0)
    dPre = (dZ @ W2) * gelu_grad(pre)
    gW1 = dPre.T @ X
    gb1 = dPre.sum(axis=0)
    return loss, dict(W1=gW1, b1=gb1, W2=gW2, b2=gb2)


def adam_step(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
