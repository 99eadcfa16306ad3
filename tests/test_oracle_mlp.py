"""Pins for the oracle MLP: reverse-mode gradients against central finite
differences, the Adam update against its published definition worked by
hand for scalars, and the linear regime (all pre-activations positive) where
the network is an affine map with a closed-form gradient."""
import numpy as np
import pytest

import synth
from oracle import mlp

rng = np.random.default_rng(11)


def _net(sizes=(7, 5, 4, 3), seed=1):
    params = synth.mlp_init(list(sizes), seed)
    params = [p + 0.1 * rng.normal(size=p.shape) for p in params]  # non-zero biases
    X = rng.normal(size=(6, sizes[0]))
    T = rng.normal(size=(6, sizes[-1]))
    return params, X, T


def test_gradients_match_finite_differences():
    params, X, T = _net()
    g = mlp.gradients(params, X, T)
    eps = 1e-6
    for k, p in enumerate(params):
        flat = p.ravel()
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            plus = [q.copy() for q in params]
            minus = [q.copy() for q in params]
            plus[k].ravel()[idx] += eps
            minus[k].ravel()[idx] -= eps
            fd = (mlp.loss(plus, X, T) - mlp.loss(minus, X, T)) / (2 * eps)
            assert g[k].ravel()[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_steps_by_hand():
    # scalar parameter 1.0, gradients 0.5 then -0.25, lr 0.1, default betas
    p = [np.array(1.0)]
    m = [np.array(0.0)]
    v = [np.array(0.0)]
    p, m, v = mlp.adam_step(p, [np.array(0.5)], m, v, 1, lr=0.1)
    # m = 0.05, v = 0.00025; mhat = 0.5, vhat = 0.25 -> step 0.1 * 0.5 / (0.5 + 1e-8)
    assert m[0] == pytest.approx(0.05)
    assert v[0] == pytest.approx(0.00025)
    assert p[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8), rel=1e-15)
    p, m, v = mlp.adam_step(p, [np.array(-0.25)], m, v, 2, lr=0.1)
    m2 = 0.9 * 0.05 + 0.1 * -0.25
    v2 = 0.999 * 0.00025 + 0.001 * 0.0625
    step = 0.1 * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert m[0] == pytest.approx(m2)
    assert p[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8) - step, rel=1e-14)


def test_linear_regime_closed_form():
    """With non-negative inputs and weights and positive biases every ReLU is
    active, so y = X A^T + c with A = W3 W2 W1 and the loss gradient w.r.t. b3
    is mean(y - t)."""
    sizes = [4, 3, 3, 2]
    params = [np.abs(p) + 0.1 for p in synth.mlp_init(sizes, 2)]
    X = np.abs(rng.normal(size=(5, 4)))
    T = rng.normal(size=(5, 2))
    W1, b1, W2, b2, W3, b3 = params
    A = W3 @ W2 @ W1
    c = W3 @ (W2 @ b1 + b2) + b3
    y, _ = mlp.forward(params, X)
    assert np.allclose(y, X @ A.T + c, atol=1e-12)
    g = mlp.gradients(params, X, T)
    assert np.allclose(g[5], (y - T).mean(axis=0), atol=1e-12)
