"""The modal moment-fitting cubature (Sec. 3.8, Alg. 3), host-side setup:
moment conditions, sparsity, non-negativity and exactness of the degree-2
integrals of the basis functions (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from paper_2508_13386_gb300 import basis, cubature


@pytest.fixture(scope="module")
def beam():
    s = synth.beam_scene(material_seed=4)
    B = basis.build_sms_basis(s.X, s.tets, s.E, 32, dirichlet=s.dirichlet, seed=1)
    C = cubature.build_cubature(s.X, s.tets, B, seed=0, workers=1)
    return s, B, C


def _vol(s):
    D = np.stack([s.X[s.tets[:, k]] - s.X[s.tets[:, 0]] for k in (1, 2, 3)], axis=-1)
    return np.linalg.det(D) / 6.0


def test_moment_conditions_and_weights(beam):
    s, B, C = beam
    assert C["residual"].max() <= cubature.DEFAULT_TOL
    assert np.all(C["weight"] > 0)
    assert np.all(np.diff(C["elem"]) > 0)                      # sorted, each element once
    assert len(C["elem"]) < len(s.tets) // 4                    # sparse
    assert np.all(C["points"] <= C["constraints"])              # NNLS: at most m_P points
    vol = _vol(s)
    on = np.zeros(len(s.tets), bool)
    on[C["elem"]] = True
    assert np.allclose(C["scale"][on], C["weight"] / vol[on], rtol=1e-15)
    assert np.all(C["scale"][~on] == 0)


def test_degree_two_integrals_exact_over_the_mesh(beam):
    """Independent of the per-partition matrices: with the tet-averaged
    weights u (t x m), the cubature reproduces the whole mesh's volume,
    every integral of u_i and every integral of u_i u_j to the fitting
    tolerance (the partitions' conditions add up to these)."""
    s, B, C = beam
    m = len(B["origins"])
    n = len(s.X)
    Phi = sp.csr_matrix((B["phi"], B["handle"], B["vrow"]), shape=(n, m)).toarray()
    u = Phi[s.tets].mean(axis=1)                                # [t, m]
    vol = _vol(s)
    w = C["scale"] * vol
    assert w.sum() == pytest.approx(vol.sum(), rel=1e-9)
    assert np.allclose(u.T @ w, u.T @ vol, rtol=0, atol=1e-9 * vol.sum())
    G_full = u.T @ (vol[:, None] * u)
    G_cub = u.T @ (w[:, None] * u)
    assert np.abs(G_cub - G_full).max() <= 1e-9 * np.abs(G_full).max() * 10


def test_constant_function_needs_one_point():
    """One handle with weight 1 everywhere: the constraints 1, u, u^2 are
    one functional (rank 1), so one element carries the whole volume."""
    s = synth.tiny_scene(4, 3, 2, seed=3)
    n, t = len(s.X), len(s.tets)
    B = {"origins": s.X[:1], "vrow": np.arange(n + 1, dtype=np.int32), "handle": np.zeros(n, np.int32),
         "phi": np.ones(n), "partition": np.zeros(t, np.int64)}
    C = cubature.build_cubature(s.X, s.tets, B, seed=5, workers=1)
    assert len(C["elem"]) == 1
    assert C["weight"][0] == pytest.approx(_vol(s).sum(), rel=1e-12)
    assert C["constraints"][0] == 3


def test_seeded_and_repeatable(beam):
    s, B, C = beam
    C2 = cubature.build_cubature(s.X, s.tets, B, seed=0, workers=1)
    assert np.array_equal(C["elem"], C2["elem"]) and np.array_equal(C["weight"], C2["weight"])


def test_moment_matrix_rows():
    """Rows of A for two functions: 1, u0, u1, u0^2, u0 u1, u1^2."""
    U = np.array([[0.5, 0.25], [1.0, 0.0], [0.2, 0.8]])
    A = cubature.moment_matrix(U)
    expect = np.array([[1, 1, 1], [0.5, 1.0, 0.2], [0.25, 0.0, 0.8], [0.25, 1.0, 0.04],
                       [0.125, 0.0, 0.16], [0.0625, 0.0, 0.64]])
    assert np.allclose(A, expect, rtol=0, atol=1e-15)
