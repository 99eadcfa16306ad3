"""Pins for the oracle's Neo-Hookean element model (no GPU).

Each check is fixed by mathematics, not by re-running the oracle's own
formula: finite differences, rotation invariance, the closed-form uniaxial
stretch, the textbook linear-elastic tensor at rest, the rigid null space,
and a symbolic derivative taken independently by sympy.
"""
import numpy as np
import pytest

from oracle import elastic
import synth

rng = np.random.default_rng(1234)


def random_F(n, scale=0.2):
    F = np.eye(3)[None] + scale * rng.normal(size=(n, 3, 3))
    det = np.linalg.det(F)
    F[det < 0, :, 0] *= -1.0
    return F


def random_rotation():
    Q, R = np.linalg.qr(rng.normal(size=(3, 3)))
    Q = Q * np.sign(np.diag(R))[None, :]
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def test_rest_state_has_zero_energy_and_stress():
    mu, lam = elastic.lame(np.array([1e5, 1e9]), np.array([0.45, 0.3]))
    F = np.stack([np.eye(3)] * 2)
    assert np.allclose(elastic.psi(F, mu, lam), 0.0, atol=1e-12)
    assert np.allclose(elastic.first_pk(F, mu, lam), 0.0, atol=1e-6)


def test_lame_parameters_textbook():
    mu, lam = elastic.lame(2.6, 0.3)
    assert mu == pytest.approx(1.0)
    assert lam == pytest.approx(2.6 * 0.3 / (1.3 * 0.4))


def test_uniaxial_stretch_closed_form():
    mu, lam = 3.0, 7.0
    for s in [0.5, 0.9, 1.0, 1.3, 2.0]:
        F = np.diag([s, 1.0, 1.0])[None]
        expect = mu / 2 * (s * s - 1) - mu * np.log(s) + lam / 2 * np.log(s) ** 2
        assert elastic.psi(F, mu, lam)[0] == pytest.approx(expect, rel=1e-14, abs=1e-14)


def test_inverted_is_infinite():
    F = np.diag([-1.0, 1.0, 1.0])[None]
    assert np.isinf(elastic.psi(F, 1.0, 1.0)[0])


def test_rotation_invariance():
    F = random_F(20)
    mu = rng.uniform(1, 10, 20)
    lam = rng.uniform(1, 10, 20)
    R = random_rotation()
    a = elastic.psi(F, mu, lam)
    b = elastic.psi(R[None] @ F, mu, lam)
    assert np.allclose(a, b, rtol=1e-12)


def test_first_pk_matches_finite_differences():
    F = random_F(5)
    mu = rng.uniform(1, 10, 5)
    lam = rng.uniform(1, 10, 5)
    P = elastic.first_pk(F, mu, lam)
    eps = 1e-6
    for a in range(3):
        for b in range(3):
            dF = np.zeros((3, 3))
            dF[a, b] = eps
            fd = (elastic.psi(F + dF, mu, lam) - elastic.psi(F - dF, mu, lam)) / (2 * eps)
            assert np.allclose(P[:, a, b], fd, rtol=1e-7, atol=1e-7)


def test_stress_derivative_matches_finite_differences():
    F = random_F(5)
    mu = rng.uniform(1, 10, 5)
    lam = rng.uniform(1, 10, 5)
    D = elastic.stress_derivative(F, mu, lam)
    eps = 1e-6
    for k in range(3):
        for l in range(3):
            dF = np.zeros((3, 3))
            dF[k, l] = eps
            fd = (elastic.first_pk(F + dF, mu, lam) - elastic.first_pk(F - dF, mu, lam)) / (2 * eps)
            assert np.allclose(D[:, :, 3 * k + l], fd.reshape(5, 9), rtol=1e-6, atol=1e-6)


def test_stress_derivative_symbolic():
    sympy = pytest.importorskip("sympy")
    Fs = sympy.Matrix(3, 3, sympy.symbols("f0:9"))
    mu_s, lam_s = sympy.symbols("mu lam", positive=True)
    J = Fs.det()
    psi = mu_s / 2 * (sum(v * v for v in Fs) - 3) - mu_s * sympy.log(J) + lam_s / 2 * sympy.log(J) ** 2
    flat = list(Fs)
    F = random_F(1)[0]
    subs = {s: float(v) for s, v in zip(flat, F.ravel())}
    subs[mu_s] = 2.5
    subs[lam_s] = 4.0
    grad = [sympy.diff(psi, s) for s in flat]
    P_sym = np.array([float(g.evalf(subs=subs)) for g in grad])
    D_sym = np.array([[float(sympy.diff(g, s).evalf(subs=subs)) for s in flat] for g in grad])
    P = elastic.first_pk(F[None], np.array([2.5]), np.array([4.0]))[0].ravel()
    D = elastic.stress_derivative(F[None], np.array([2.5]), np.array([4.0]))[0]
    assert np.allclose(P, P_sym, rtol=1e-12, atol=1e-12)
    assert np.allclose(D, D_sym, rtol=1e-12, atol=1e-12)


def test_rest_stress_derivative_is_linear_elastic_tensor():
    mu, lam = 3.0, 5.0
    D = elastic.stress_derivative(np.eye(3)[None], np.array([mu]), np.array([lam]))[0]
    d = np.eye(3)
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = mu * (d[i, k] * d[j, l] + d[i, l] * d[j, k]) + lam * d[i, j] * d[k, l]
    assert np.allclose(D, C.reshape(9, 9), atol=1e-12)


def test_dFdx_reproduces_affine_maps():
    mesh = synth.random_tet_mesh(2, 2, 1, seed=3)
    vol, Dm_inv = elastic.rest_shape(mesh.X, mesh.tets)
    A = rng.normal(size=(3, 3))
    t = rng.normal(size=3)
    x = mesh.X @ A.T + t
    B = elastic.dF_dx(Dm_inv)
    xe = x[mesh.tets].reshape(-1, 12)
    F_vec = np.einsum("tri,ti->tr", B, xe)
    assert np.allclose(F_vec, np.broadcast_to(A.ravel(), F_vec.shape), atol=1e-12)
    assert np.allclose(elastic.deformation_gradient(x, mesh.tets, Dm_inv), A[None], atol=1e-12)


def _tiny():
    s = synth.tiny_scene(2, 1, 1, seed=5)
    vol, Dm_inv = elastic.rest_shape(s.X, s.tets)
    mu, lam = elastic.lame(s.E, s.nu)
    x = s.X + 0.01 * rng.normal(size=s.X.shape)
    return s, vol, Dm_inv, mu, lam, x


def test_element_gradient_matches_finite_differences():
    s, vol, Dm_inv, mu, lam, x = _tiny()
    g = elastic.element_gradient(x, s.tets, vol, Dm_inv, mu, lam)
    eps = 1e-7
    for e in range(3):
        for i in range(12):
            v, c = s.tets[e, i // 3], i % 3
            xp = x.copy(); xp[v, c] += eps
            xm = x.copy(); xm[v, c] -= eps
            fd = (elastic.element_energy(xp, s.tets, vol, Dm_inv, mu, lam)[e]
                  - elastic.element_energy(xm, s.tets, vol, Dm_inv, mu, lam)[e]) / (2 * eps)
            assert fd == pytest.approx(g[e, i], rel=1e-5, abs=1e-6 * np.abs(g[e]).max())


def test_unprojected_element_hessian_matches_finite_differences():
    s, vol, Dm_inv, mu, lam, x = _tiny()
    H = elastic.element_hessian(x, s.tets, vol, Dm_inv, mu, lam, project=False)
    eps = 1e-7
    for e in range(2):
        for i in range(12):
            v, c = s.tets[e, i // 3], i % 3
            xp = x.copy(); xp[v, c] += eps
            xm = x.copy(); xm[v, c] -= eps
            fd = (elastic.element_gradient(xp, s.tets, vol, Dm_inv, mu, lam)[e]
                  - elastic.element_gradient(xm, s.tets, vol, Dm_inv, mu, lam)[e]) / (2 * eps)
            assert np.allclose(H[e, :, i], fd, rtol=1e-5, atol=1e-5 * np.abs(H[e]).max())


def test_rest_hessian_has_rigid_null_space():
    s, vol, Dm_inv, mu, lam, _ = _tiny()
    H = elastic.element_hessian(s.X, s.tets, vol, Dm_inv, mu, lam, project=True)
    for e in range(len(s.tets)):
        Xe = s.X[s.tets[e]]
        modes = []
        for c in range(3):
            t = np.zeros((4, 3)); t[:, c] = 1.0
            modes.append(t.ravel())
        for axis in np.eye(3):
            modes.append(np.cross(axis[None, :], Xe).ravel())
        for m in modes:
            assert np.linalg.norm(H[e] @ m) <= 1e-9 * np.linalg.norm(H[e]) * np.linalg.norm(m)
        w = np.linalg.eigvalsh(H[e])
        assert np.sum(w > 1e-9 * w.max()) == 6


def test_psd_project_properties():
    A = rng.normal(size=(10, 9, 9))
    A = A + np.swapaxes(A, 1, 2)
    P = elastic.psd_project(A)
    assert np.all(np.linalg.eigvalsh(P) >= -1e-12 * np.abs(A).max())
    S = A @ np.swapaxes(A, 1, 2)
    assert np.allclose(elastic.psd_project(S), S, atol=1e-10)
    M = np.diag([3.0, -2.0])[None]
    assert np.allclose(elastic.psd_project(M)[0], np.diag([3.0, 0.0]))


def test_projected_hessian_is_psd_under_compression():
    s, vol, Dm_inv, mu, lam, _ = _tiny()
    x = s.X * np.array([0.6, 1.0, 1.0])[None, :]
    Hu = elastic.element_hessian(x, s.tets, vol, Dm_inv, mu, lam, project=False)
    Hp = elastic.element_hessian(x, s.tets, vol, Dm_inv, mu, lam, project=True)
    assert np.min(np.linalg.eigvalsh(Hu)) < 0
    assert np.min(np.linalg.eigvalsh(Hp)) >= -1e-9 * np.abs(Hp).max()
