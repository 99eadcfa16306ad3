"""CPU checks of the C ABI boundary: the library loads without a GPU, exports
every entry point declared in include/mls.h, and the binding refuses to run
without it."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mls.h")).read()
    return set(re.findall(r"^(?:mls_status|const char\*|int64_t|double)\s+(mls_\w+)\(", text, re.M))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_13386_gb300 import _lib
    lib = _lib.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert _declared() == set(_lib.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mls_\w+)", out))
    assert _declared() <= exported


def test_missing_library_fails_loudly(tmp_path):
    from paper_2508_13386_gb300 import _lib
    with pytest.raises(ImportError, match="build the CUDA library"):
        _lib.load(str(tmp_path / "libmls.so"))


def test_options_roundtrip_on_cpu():
    import ctypes as C
    from paper_2508_13386_gb300 import _lib
    lib = _lib.load()
    o = _lib.Options()
    assert lib.mls_default_options(C.byref(o)) == 0
    assert o.precision == 0 and o.pcg_rtol == 1e-4 and o.max_newton == 50
    assert lib.mls_default_options(None) == -1


def test_tridiagonal_max_eigenvalue_matches_dense_solver():
    """The Sturm-bisection bound behind the automatic smoother damping
    (host code, no GPU): against numpy's dense eigenvalues for random,
    clustered, split (zero off-diagonal) and 1 x 1 tridiagonals."""
    import numpy as np
    import paper_2508_13386_gb300 as mls
    rng = np.random.default_rng(7)
    cases = [(np.array([2.5]), np.zeros(0))]
    for k in (2, 5, 20, 40):
        cases.append((rng.normal(size=k) * 3, rng.normal(size=k - 1)))
        cases.append((np.full(k, 2.0) + 1e-9 * rng.normal(size=k), np.full(k - 1, 1.0)))
        e = rng.normal(size=k - 1)
        e[k // 2 - 1] = 0.0
        cases.append((rng.uniform(0.1, 3.0, size=k), e))
    for d, e in cases:
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        lam = np.linalg.eigvalsh(T).max()
        got = mls.tridiag_max_eig(d, e)
        scale = np.abs(T).max()
        assert got >= lam - 1e-13 * scale and got - lam <= 1e-12 * scale, (got, lam)
    assert np.isnan(mls.tridiag_max_eig(np.zeros(0), np.zeros(0)))
