"""Shared helpers for the GPU parity tests (CUDA path vs the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=cuda())


def host(t):
    return t.detach().cpu().numpy()


def solver_for(scene, **opts):
    import paper_2508_13386_gb300 as mls
    s = mls.Solver(**opts)
    s.setup_scene(scene)
    return s


def rel_disp_error(x_gpu, x_orc, x_t):
    """Per-step relative displacement error |x_gpu - x_orc| / |x_orc - x^t|."""
    return float(np.linalg.norm(x_gpu - x_orc) / max(np.linalg.norm(x_orc - x_t), 1e-300))
