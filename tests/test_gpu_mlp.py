"""Parity of the learned-model kernels (forward, gradients, Adam, training)
against the FP64 oracle MLP.

The GPU multiplies BF16 operands with FP32 accumulation on the tensor
cores.  The checks emulate exactly the roundings the kernels make: weights,
inputs and hidden activations are rounded to BF16 before each product, and
in the backward pass so are the back-propagated errors dY, dZ2 and dZ1
before they enter a product (bias gradients sum the FP32 errors).  What
remains is FP32-vs-FP64 accumulation (relative ~1e-7) and, rarely, a BF16
rounding that goes the other way: an intermediate that lies within that
accumulation error of a BF16 rounding boundary changes by one BF16 ulp
(2^-8 relative), and everything downstream of it moves.  In the small
network no rounding flips and the forward outputs agree to 1e-5 of the
largest; at the configured widths the 1152-term sums carry ~3e-6 of
accumulation error, about one hidden unit in a thousand flips, and each
flip moves its sample's whole output row, so the forward pass is held to
2e-3 in Frobenius norm.  Per parameter block the gradients agree to 5e-3
(a flip in a back-propagated error moves a whole row of a weight
gradient).  The sizes are a small network (several tiles, ragged edges)
and the configured one, 1152 -> 256 -> 256 -> 384.  Adam is elementwise
FP32: relative 1e-5.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import mlp as omlp

from gpu_helpers import torch

pytestmark = pytest.mark.gpu

SIZES = [96, 64, 64, 40]
FULL = [1152, 256, 256, 384]


def bf16(a):
    """Round to bfloat16 (nearest even) and back, as the kernels do."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def flat(params):
    return np.concatenate([p.ravel() for p in params]).astype(np.float32)


def unflat(vec, sizes):
    out, k = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        out.append(vec[k:k + fo * fi].reshape(fo, fi)); k += fo * fi
        out.append(vec[k:k + fo]); k += fo
    return out


def make(sizes, batch, seed=0):
    import paper_2508_13386_gb300 as mls
    lib = mls._get_lib()
    params = synth.mlp_init(sizes, seed)
    params = [p + (0.05 if p.ndim == 1 else 0.0) for p in params]
    init = flat(params)
    h = C.c_void_p()
    st = lib.mls_mlp_create(C.byref(h), sizes[0], sizes[1], sizes[3], batch,
                            init.ctypes.data_as(C.c_void_p), None)
    assert st == 0
    return lib, h, unflat(init.astype(np.float64), sizes)


def ptr(t):
    return C.c_void_p(t.data_ptr())


def emulated_gradients(params, X, T, rnd=None):
    """The oracle's back-propagation (oracle.mlp.gradients) with the BF16
    roundings of the kernels' operands: weights, input, hidden activations
    and back-propagated errors enter each product rounded by rnd (BF16)."""
    bf16 = rnd if rnd is not None else globals()["bf16"]
    W1, b1, W2, b2, W3, b3 = params
    Wb1, Wb2, Wb3 = bf16(W1), bf16(W2), bf16(W3)
    Xb = bf16(X)
    B = X.shape[0]
    h1 = np.maximum(Xb @ Wb1.T + b1, 0)
    h2 = np.maximum(bf16(h1) @ Wb2.T + b2, 0)
    y = bf16(h2) @ Wb3.T + b3
    dy = (y - T) / B
    dW3 = bf16(dy).T @ bf16(h2)
    d2 = (bf16(dy) @ Wb3) * (h2 > 0)
    dW2 = bf16(d2).T @ bf16(h1)
    d1 = (bf16(d2) @ Wb2) * (h1 > 0)
    dW1 = bf16(d1).T @ Xb
    loss = 0.5 * np.sum((y - T) ** 2) / B
    return [dW1, d1.sum(0), dW2, d2.sum(0), dW3, dy.sum(0)], loss


def test_bf16_emulation_reduces_to_the_oracle():
    """The emulation is the oracle's gradient with roundings inserted: with
    the identity in place of the BF16 rounding it reproduces
    oracle.mlp.gradients and oracle.mlp.loss."""
    rng = np.random.default_rng(7)
    params = [p + 0.05 * (p.ndim == 1) for p in synth.mlp_init(SIZES, 3)]
    X = rng.normal(size=(12, SIZES[0]))
    T = rng.normal(size=(12, SIZES[3]))
    g, loss = emulated_gradients(params, X, T, rnd=lambda a: np.asarray(a, dtype=np.float64))
    for a, b in zip(g, omlp.gradients(params, X, T)):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14)
    assert loss == pytest.approx(omlp.loss(params, X, T), rel=1e-12)


@pytest.mark.parametrize("sizes,n", [(SIZES, 150), (FULL, 300)])
def test_forward_matches_bf16_emulated_oracle(sizes, n):
    lib, h, params = make(sizes, 64 if sizes is SIZES else 256)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(n, sizes[0])).astype(np.float32)   # several tiles + ragged tail
    Xd = torch.as_tensor(X, device="cuda:0")
    Yd = torch.empty(n, sizes[3], dtype=torch.float32, device="cuda:0")
    assert lib.mls_mlp_forward(h, ptr(Xd), n, ptr(Yd)) == 0
    W1, b1, W2, b2, W3, b3 = params
    h1 = np.maximum(bf16(X) @ bf16(W1).T + b1, 0)
    h2 = np.maximum(bf16(h1) @ bf16(W2).T + b2, 0)
    y = bf16(h2) @ bf16(W3).T + b3
    Y = Yd.cpu().numpy()
    if sizes is SIZES:
        assert np.max(np.abs(Y - y)) <= 1e-5 * np.abs(y).max()
    assert np.linalg.norm(Y - y) <= 2e-3 * np.linalg.norm(y)
    lib.mls_mlp_destroy(h)


@pytest.mark.parametrize("sizes,batch", [(SIZES, 48), (SIZES, 37), (FULL, 256)])
def test_gradients_match_oracle(sizes, batch):
    lib, h, params = make(sizes, batch)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(batch, sizes[0])).astype(np.float32)
    T = rng.normal(size=(batch, sizes[3])).astype(np.float32)
    P = lib.mls_mlp_param_count(h)
    G = torch.empty(P, dtype=torch.float32, device="cuda:0")
    loss = C.c_double()
    assert lib.mls_mlp_gradients(h, ptr(torch.as_tensor(X, device="cuda:0")),
                                 ptr(torch.as_tensor(T, device="cuda:0")), batch, ptr(G), C.byref(loss)) == 0
    g_o, loss_o = emulated_gradients(params, X.astype(np.float64), T.astype(np.float64))
    g = unflat(G.cpu().numpy().astype(np.float64), sizes)
    for a, b in zip(g, g_o):
        assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b)
    assert loss.value == pytest.approx(loss_o, rel=1e-4)
    lib.mls_mlp_destroy(h)


def test_adam_step_matches_oracle():
    lib, h, params = make(SIZES, 16)
    rng = np.random.default_rng(3)
    P = lib.mls_mlp_param_count(h)
    grads = [rng.normal(size=p.shape) for p in params]
    G = torch.as_tensor(flat(grads), device="cuda:0")
    zeros = [np.zeros_like(p) for p in params]
    p_o, m_o, v_o = omlp.adam_step(params, [g.astype(np.float32).astype(np.float64) for g in grads], zeros, zeros,
                                   1, lr=1e-2)
    p_o, m_o, v_o = omlp.adam_step(p_o, [g.astype(np.float32).astype(np.float64) for g in grads], m_o, v_o, 2, lr=1e-2)
    assert lib.mls_mlp_adam_step(h, ptr(G), C.c_float(1e-2)) == 0
    assert lib.mls_mlp_adam_step(h, ptr(G), C.c_float(1e-2)) == 0
    out = np.zeros(P, dtype=np.float32)
    assert lib.mls_mlp_get_params(h, out.ctypes.data_as(C.c_void_p)) == 0
    ref = flat(p_o).astype(np.float64)
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.abs(ref).max()
    lib.mls_mlp_destroy(h)


def test_training_reduces_loss():
    lib, h, params = make(SIZES, 64, seed=4)
    rng = np.random.default_rng(4)
    n = 1024
    X = rng.normal(size=(n, SIZES[0])).astype(np.float32)
    A = rng.normal(size=(SIZES[3], SIZES[0])) / np.sqrt(SIZES[0])
    T = (np.tanh(X @ A.T)).astype(np.float32)
    Xd = torch.as_tensor(X, device="cuda:0")
    Td = torch.as_tensor(T, device="cuda:0")
    losses = []
    for epoch in range(30):
        order = torch.as_tensor(rng.permutation(n).astype(np.int32), device="cuda:0")
        loss = C.c_double()
        assert lib.mls_mlp_train(h, ptr(Xd), ptr(Td), n, ptr(order), n, 64, C.c_float(2e-3), C.byref(loss)) == 0
        losses.append(loss.value)
    assert losses[-1] < 0.2 * losses[0]
    lib.mls_mlp_destroy(h)
