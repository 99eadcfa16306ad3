"""The allocation-free elastic energy entry point, called through the C ABI.

It exists for callers that cannot allocate device memory while they run; its
reduction scratch is a file-scope device array.  This file is collected last
so that a failure here comes after every other test has run.  It checks the
entry point against the per-tet energies of mls_eval_elements (summed on the
host) and against the oracle's Neo-Hookean energy sum, on two calls in a row,
so that scratch left by the first call cannot leak into the second.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import elastic

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_existing_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_13386_gb300 as mls
    lib = mls._get_lib()
    dev = torch.device("cuda:0")
    s = synth.tiny_scene(7, 5, 4, seed=21)
    rng = np.random.default_rng(3)
    solver = mls.Solver(precision="fp64")
    solver.setup_scene(s)
    mu, lam = elastic.lame(s.E, s.nu)
    X = torch.as_tensor(s.X, device=dev).contiguous()
    T = torch.as_tensor(s.tets.astype(np.int32), device=dev).contiguous()
    MU = torch.as_tensor(mu, device=dev).contiguous()
    LAM = torch.as_tensor(lam, device=dev).contiguous()
    out_e = torch.zeros(1, dtype=torch.float64, device=dev)
    out_b = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    vol, Dm_inv = elastic.rest_shape(s.X, s.tets)
    for call in range(2):
        x = s.X + 0.01 * (call + 1) * rng.normal(size=s.X.shape) * 0.1
        xt = torch.as_tensor(x, device=dev).contiguous()
        E_ref, _, _ = solver.eval_elements(xt)
        ref = float(E_ref.sum())
        st = lib.mls_elastic_energy_noalloc(
            s.n_verts, s.n_tets, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), C.c_void_p(MU.data_ptr()),
            C.c_void_p(LAM.data_ptr()), C.c_void_p(xt.data_ptr()), C.c_void_p(out_e.data_ptr()),
            C.c_void_p(out_b.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        assert int(out_b.item()) == 0
        assert float(out_e.item()) == pytest.approx(ref, rel=1e-10)
        E_orc = float(elastic.element_energy(x, s.tets, vol, Dm_inv, mu, lam).sum())
        assert float(out_e.item()) == pytest.approx(E_orc, rel=1e-10)


def test_noalloc_rejects_oversized_and_null():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_13386_gb300 as mls
    lib = mls._get_lib()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    p = C.c_void_p(dummy.data_ptr())
    assert lib.mls_elastic_energy_noalloc(4, 4096 * 256 + 1, p, p, p, p, p, p, p, None) == -1
    assert lib.mls_elastic_energy_noalloc(4, 1, None, p, p, p, p, p, p, None) == -1
