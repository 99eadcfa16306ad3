"""Pins for the oracle's subspace algebra (no GPU): LBS basis layout (Eq. LBS),
linear precision under a partition of unity (Sec. 3.5), Galerkin operator
by brute force, Galerkin orthogonality, and the two-level preconditioner's
symmetry, definiteness and exactness in the full-rank case."""
import numpy as np
import pytest

import synth
from oracle import ip, pcg, subspace

rng_local = np.random.default_rng(505)

rng = np.random.default_rng(7)


def _scene_and_basis(m=5, k=3):
    s = synth.tiny_scene(3, 2, 2, seed=21, pinned=False)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=m, k=k, seed=4)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    return s, origins, vrow, handle, phi, U


def test_lbs_block_layout_single_vertex():
    X = np.array([[1.0, 2.0, 3.0]])
    origins = np.array([[0.5, 0.0, -1.0]])
    U = subspace.lbs_basis_matrix(X, origins, np.array([0, 1]), np.array([0]), np.array([0.25]))
    a = np.array([1.0, 0.5, 2.0, 4.0])
    expect = 0.25 * np.kron(np.eye(3), a[None, :])   # I_3 (x) [1, x, y, z]
    assert np.allclose(U.toarray(), expect)


def test_linear_precision_with_partition_of_unity():
    """With sum_j phi_j = 1, every affine map x -> A x + t is reproduced by
    q_j = (A o_j + t | A), the same map written about each handle origin."""
    s, origins, vrow, handle, phi, U = _scene_and_basis()
    A = rng.normal(size=(3, 3))
    t = rng.normal(size=3)
    m = origins.shape[0]
    q = np.zeros((m, 12))
    for j in range(m):
        M34 = np.concatenate([(A @ origins[j] + t)[:, None], A], axis=1)
        q[j] = M34.ravel()
    w = subspace.prolong(U, q)
    assert np.allclose(w, s.X @ A.T + t[None, :], atol=1e-12)


def test_restriction_is_transpose_of_prolongation():
    s, origins, vrow, handle, phi, U = _scene_and_basis()
    q = rng.normal(size=(origins.shape[0], 12))
    r = rng.normal(size=s.X.shape)
    lhs = np.sum(subspace.prolong(U, q) * r)
    rhs = np.sum(q * subspace.restrict(U, r))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_galerkin_brute_force():
    s, origins, vrow, handle, phi, U = _scene_and_basis(m=3, k=2)
    H = ip.Problem(s).hessian(s.X)
    Ac = subspace.galerkin(H, U)
    r = U.shape[1]
    cols = [subspace.prolong(U, np.eye(r)[a]).ravel() for a in range(r)]
    brute = np.array([[cols[a] @ (H @ cols[b]) for b in range(r)] for a in range(r)])
    assert np.allclose(Ac, brute, rtol=1e-12, atol=1e-12 * np.abs(brute).max())
    assert np.allclose(Ac, Ac.T, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
    assert np.linalg.eigvalsh(Ac).min() > 0


def test_galerkin_orthogonality():
    s, origins, vrow, handle, phi, U = _scene_and_basis()
    H = ip.Problem(s).hessian(s.X)
    Ac = subspace.galerkin(H, U)
    r = rng.normal(size=3 * s.n_verts)
    z = subspace.two_level_apply(H, U, Ac, r, mode="coarse")
    assert np.abs(U.T @ (r - H @ z)).max() <= 1e-9 * np.abs(U.T @ r).max()


@pytest.mark.parametrize("mode", ["additive", "multiplicative"])
def test_two_level_preconditioner_spd(mode):
    s, origins, vrow, handle, phi, U = _scene_and_basis()
    H = ip.Problem(s).hessian(s.X)
    Ac = subspace.galerkin(H, U)
    n3 = H.shape[0]
    M = np.stack([subspace.two_level_apply(H, U, Ac, e, mode=mode, omega=0.5)
                  for e in np.eye(n3)], axis=1)
    assert np.allclose(M, M.T, atol=1e-10 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_full_rank_coarse_space_solves_in_one_iteration():
    """When U spans the whole space the coarse correction is H^{-1}."""
    s = synth.tiny_scene(1, 1, 1, seed=3, pinned=False)
    H = ip.Problem(s).hessian(s.X)
    n3 = H.shape[0]
    import scipy.sparse as sp
    U = sp.csr_matrix(rng.normal(size=(n3, n3)))
    Ac = subspace.galerkin(H, U)
    b = rng.normal(size=n3)
    x, info = pcg.pcg(lambda v: H @ v, b,
                      lambda r: subspace.two_level_apply(H, U, Ac, r, mode="coarse"), rtol=1e-9)
    assert info["iters"] == 1


def test_multilevel_pcg_beats_jacobi_on_stiff_beam_slice():
    s = synth.tiny_scene(6, 2, 2, seed=12, pinned=True, E_range=(1e5, 1e9))
    p = ip.Problem(s)
    H = p.hessian(p.x_tilde)
    b = -p.gradient(p.x_tilde).ravel()
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=6, k=2, seed=1)
    phi = phi.copy()
    phi[np.repeat(p.pinned, 2)] = 0.0
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    Ac = subspace.galerkin(H, U)
    Ac += 1e-12 * np.trace(Ac) / Ac.shape[0] * np.eye(Ac.shape[0])
    Dinv = subspace.block_diagonal_inverse(H)
    _, jac = pcg.pcg(lambda v: H @ v, b, lambda r: Dinv @ r, rtol=1e-8)
    _, ml = pcg.pcg(lambda v: H @ v, b,
                    lambda r: subspace.two_level_apply(H, U, Ac, r, omega=0.5, Dinv=Dinv), rtol=1e-8)
    assert ml["converged"] and jac["converged"]
    assert ml["iters"] < jac["iters"]


def test_paper_direction_limits():
    """Pins of the paper-direction oracle: with U spanning the whole space
    the subspace direction is already the Newton direction and leaves no
    residual to refine; with no refinement and a one-column-block
    basis, d_s is the exact minimiser of the quadratic model in span U
    (Galerkin orthogonality U^T (g + H d_s) = 0); with many refinement
    iterations d_s + d_f is the Newton direction whatever U is."""
    import scipy.sparse as sp
    from oracle import subspace
    rng = np.random.default_rng(3)
    n3 = 36
    A = rng.normal(size=(n3, n3))
    H = sp.csr_matrix(A @ A.T + n3 * np.eye(n3))
    g = rng.normal(size=n3)
    d_newton = np.linalg.solve(H.toarray(), -g)
    full = sp.csr_matrix(np.eye(n3))
    ds, df = subspace.paper_direction(H, g, full, 0)
    assert np.allclose(ds, d_newton, rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(-g - H @ ds) <= 1e-10 * np.linalg.norm(g)   # nothing left to refine
    U = sp.csr_matrix(rng.normal(size=(n3, 12)))
    ds, df = subspace.paper_direction(H, g, U, 0)
    assert np.linalg.norm(df) == 0.0
    assert np.linalg.norm(U.T @ (g + H @ ds)) <= 1e-10 * np.linalg.norm(U.T @ g)
    ds, df = subspace.paper_direction(H, g, U, 200)
    assert np.allclose(ds + df, d_newton, rtol=1e-8, atol=1e-10)


def test_handle_block_jacobi_inverts_a_block_diagonal_matrix():
    blocks = [rng_local.normal(size=(12, 12)) for _ in range(3)]
    blocks = [b @ b.T + 12 * np.eye(12) for b in blocks]
    import scipy.sparse as sp
    A = sp.block_diag([sp.csr_matrix(b) for b in blocks]).tocsr()
    Minv = subspace.handle_block_jacobi(A)
    v = rng_local.normal(size=36)
    assert np.allclose(A @ Minv(v), v, rtol=0, atol=1e-12 * np.abs(v).max())


def test_literal_subspace_direction_reduces_to_the_galerkin_solution():
    """Alg. 2's subspace direction as printed (affine PCG, then SMS PCG on
    the residual, 12 x 12 block Jacobi, matrix-free products): when the SMS
    weights are a partition of unity the SMS space contains every affine
    motion, so solved tightly the two levels give exactly the Galerkin
    direction U_s (U_s^T H U_s)^{-1} U_s^T (-g) (the reading that an exact
    SMS solve makes the affine level redundant).  At the paper's 1e-4 the
    SMS level meets its own residual criterion."""
    s = synth.tiny_scene(6, 4, 3, seed=15, E_range=(1e5, 1e8))
    p = ip.Problem(s)
    H = p.hessian(p.x_tilde)
    g = p.gradient(p.x_tilde).ravel()
    o, vr, h, ph = synth.random_sparse_basis(s.X, m=7, k=3, seed=3)
    Us = subspace.lbs_basis_matrix(s.X, o, vr, h, ph)
    _, Ua = subspace.affine_basis_matrix(s.X, mass=p.mass)
    ref = Us @ subspace.coarse_solve(subspace.galerkin(H, Us), Us.T @ (-g))
    ds, (ia, is_) = subspace.subspace_direction_literal(H, g, Ua, Us, rtol=1e-12)
    assert np.linalg.norm(ds - ref) <= 1e-9 * np.linalg.norm(ref)
    assert ia == 1                      # one object: the 12 x 12 block preconditioner is exact
    ds4, _ = subspace.subspace_direction_literal(H, g, Ua, Us, rtol=1e-4)
    r_before = Us.T @ (-g - H @ (Ua @ subspace.coarse_solve(subspace.galerkin(H, Ua), Ua.T @ (-g))))
    r_after = Us.T @ (-g - H @ ds4)
    assert np.linalg.norm(r_after) <= 1e-4 * np.linalg.norm(r_before) * (1 + 1e-6)
