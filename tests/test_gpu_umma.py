"""The tensor-core product C = A B^T (bf16 operands staged by TMA, tcgen05
with a float32 accumulator in tensor memory), called through the C ABI.

Reference: the float64 product of the same bf16 values in numpy.  Products of
bf16 values are exact in float32, so the only error is float32 accumulation:
|C - C_ref| <= K 2^-23 sum_k |a_ik b_jk| per element, checked with a margin.
Shapes cover one tile, ragged edges in M, N and K (rows and columns past
the ends read as zero), and more K blocks than the four pipeline stages.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bf16(t):
    import torch
    return t.to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 200), (256, 384, 1152), (40, 1920, 256),
                                   (7, 9, 8)])
def test_gemm_matches_float64_product(M, N, K):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_13386_gb300 as mls
    lib = mls._get_lib()
    dev = torch.device("cuda:0")
    g = torch.Generator().manual_seed(M * 7919 + N * 31 + K)
    A = _bf16(torch.randn(M, K, generator=g)).to(dev)
    B = _bf16(torch.randn(N, K, generator=g)).to(dev)
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    st = lib.mls_gemm_bf16(M, N, K, C.c_void_p(A.data_ptr()), K, C.c_void_p(B.data_ptr()), K,
                           C.c_void_p(Cd.data_ptr()), N, None)
    assert st == 0
    a = A.float().cpu().numpy().astype(np.float64)
    b = B.float().cpu().numpy().astype(np.float64)
    ref = a @ b.T
    bound = K * 2.0 ** -23 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(Cd.cpu().numpy().astype(np.float64) - ref)
    assert np.all(np.isfinite(Cd.cpu().numpy()))
    assert np.all(err <= 2 * bound), float(np.max(err / bound))


def test_gemm_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_13386_gb300 as mls
    lib = mls._get_lib()
    A = torch.zeros(16, 16, dtype=torch.bfloat16, device="cuda:0")
    Cd = torch.zeros(16, 16, dtype=torch.float32, device="cuda:0")
    p = C.c_void_p(A.data_ptr())
    c = C.c_void_p(Cd.data_ptr())
    assert lib.mls_gemm_bf16(16, 16, 16, p, 12, p, 16, c, 16, None) == -1   # lda not a multiple of 8
    assert lib.mls_gemm_bf16(16, 16, 16, p, 16, p, 16, c, 8, None) == -1    # ldc < N
    assert lib.mls_gemm_bf16(0, 16, 16, p, 16, p, 16, c, 16, None) == -1
