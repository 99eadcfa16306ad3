"""FP64 multilayer perceptron, its gradient and the Adam update (oracle).

The learned warm start maps features of the coarse (subspace) state to the
coarse increment of the timestep with a 3-layer MLP of width 256 (ReLU
hidden activations, linear output):

    h1 = relu(x W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3,

weights W_k stored [out, in].  Training minimises the mean squared error
L = 1/(2B) sum_b |y_b - t_b|^2 over a batch of B samples with Adam
(Kingma & Ba, 2015):
    m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
    w <- w - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).
Initial weights are inputs (drawn by ``synth.mlp_init``).
"""
from __future__ import annotations

import numpy as np


def forward(params, X):
    """Returns (y, cache) for a batch X [B, in]."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss(params, X, T):
    y, _ = forward(params, X)
    return 0.5 * np.sum((y - T) ** 2) / X.shape[0]


def gradients(params, X, T):
    """dL/d(params) by reverse-mode differentiation of the network."""
    W1, b1, W2, b2, W3, b3 = params
    y, (X, z1, h1, z2, h2) = forward(params, X)
    B = X.shape[0]
    dy = (y - T) / B
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, k, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step k (1-based); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = beta1 * mm + (1 - beta1) * g
        vv = beta2 * vv + (1 - beta2) * g * g
        mhat = mm / (1 - beta1 ** k)
        vhat = vv / (1 - beta2 ** k)
        out_p.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
