"""Parity of the learned-model kernels (forward, gradients, Adam, training)
against the FP64 oracle MLP.

The GPU multiplies BF16 operands with FP32 accumulation.  The forward check
emulates exactly the roundings the kernels make (weights, inputs and hidden
activations rounded to BF16 before each product), leaving only FP32-vs-FP64
accumulation: relative 1e-5.  Gradients additionally round the
back-propagated errors to BF16 when they enter a product, which the oracle
does not emulate: relative 2e-2 per parameter block.  Adam is elementwise
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


def test_forward_matches_bf16_emulated_oracle():
    lib, h, params = make(SIZES, 64)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(150, SIZES[0])).astype(np.float32)   # several tiles + ragged tail
    Xd = torch.as_tensor(X, device="cuda:0")
    Yd = torch.empty(150, SIZES[3], dtype=torch.float32, device="cuda:0")
    assert lib.mls_mlp_forward(h, ptr(Xd), 150, ptr(Yd)) == 0
    W1, b1, W2, b2, W3, b3 = params
    h1 = np.maximum(bf16(X) @ bf16(W1).T + b1, 0)
    h2 = np.maximum(bf16(h1) @ bf16(W2).T + b2, 0)
    y = bf16(h2) @ bf16(W3).T + b3
    Y = Yd.cpu().numpy()
    assert np.max(np.abs(Y - y)) <= 1e-5 * np.abs(y).max()
    lib.mls_mlp_destroy(h)


def test_gradients_match_oracle():
    lib, h, params = make(SIZES, 48)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(48, SIZES[0])).astype(np.float32)
    T = rng.normal(size=(48, SIZES[3])).astype(np.float32)
    P = lib.mls_mlp_param_count(h)
    G = torch.empty(P, dtype=torch.float32, device="cuda:0")
    loss = C.c_double()
    assert lib.mls_mlp_gradients(h, ptr(torch.as_tensor(X, device="cuda:0")),
                                 ptr(torch.as_tensor(T, device="cuda:0")), 48, ptr(G), C.byref(loss)) == 0
    bparams = [bf16(p) if p.ndim == 2 else p for p in params]
    g_o = omlp.gradients(bparams, bf16(X), T.astype(np.float64))
    g = unflat(G.cpu().numpy().astype(np.float64), SIZES)
    for a, b in zip(g, g_o):
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b)
    assert loss.value == pytest.approx(omlp.loss(bparams, bf16(X), T.astype(np.float64)), rel=2e-2)
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
