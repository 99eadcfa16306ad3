"""Pins for the oracle's lagged, mollified point-plane friction (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import barrier, friction, ip, newton

rng = np.random.default_rng(11)


def test_mollifier_closed_forms():
    eps = 2e-3
    y = np.array([0.0, 0.5 * eps, eps, 3 * eps])
    assert np.allclose(friction.f0(y, eps), [eps / 3, -eps / 24 + eps / 4 + eps / 3, eps, 3 * eps], rtol=1e-15)
    assert np.allclose(friction.f1(y, eps), [0.0, 0.75, 1.0, 1.0], rtol=1e-15)
    # f0' = f1 and f1' = df1 (central differences), f1' >= 0
    ys = np.linspace(1e-5, 2 * eps, 41)
    dy = 1e-9
    assert np.allclose((friction.f0(ys + dy, eps) - friction.f0(ys - dy, eps)) / (2 * dy),
                       friction.f1(ys, eps), rtol=1e-6, atol=1e-8)
    inner = ys[ys < eps - 2 * dy]
    assert np.allclose((friction.f1(inner + dy, eps) - friction.f1(inner - dy, eps)) / (2 * dy),
                       friction.df1(inner, eps), rtol=1e-6, atol=1e-6 / eps)
    assert np.all(friction.df1(ys, eps) >= 0)


def test_tangent_basis_is_orthonormal_and_tangent():
    for n in ([0, 0, 1], [1, 0, 0], [0.3, -0.4, 0.8]):
        n = np.asarray(n, float) / np.linalg.norm(n)
        T = friction.tangent_basis(n)
        assert np.allclose(T.T @ T, np.eye(2), atol=1e-15)
        assert np.allclose(n @ T, 0, atol=1e-15)


def _contact_state(n_vert=12, sliding=False):
    dhat, kappa, h = 1e-3, 1e5, 1.0 / 60
    x_t = rng.uniform(-1, 1, size=(n_vert, 3))
    x_t[:, 2] = rng.uniform(1e-4, 2e-3, size=n_vert)          # some within dhat, some outside
    du = (rng.normal(size=(n_vert, 3)) * (5e-3 if sliding else 1e-5))
    return x_t, x_t + du, dhat, kappa, h


@pytest.mark.parametrize("sliding", [False, True])
def test_friction_derivatives_match_finite_differences(sliding):
    x_t, x, dhat, kappa, h = _contact_state(sliding=sliding)
    F = friction.GroundFriction(0.4, 1e-3, h, kappa, dhat, [0, 0, 1], 0.0, x_t)
    assert np.any(F.lam > 0) and np.any(F.lam == 0)
    g = F.gradient(x)
    H = F.hessian_blocks(x)
    e = 1e-9
    for v in np.nonzero(F.lam > 0)[0][:5]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += e
            xm[v, c] -= e
            fd = (F.energy(xp) - F.energy(xm)) / (2 * e)
            assert fd == pytest.approx(g[v, c], rel=1e-5, abs=1e-6 * np.abs(g).max())
            fdg = (F.gradient(xp)[v] - F.gradient(xm)[v]) / (2 * e)
            assert np.allclose(fdg, H[v, :, c], rtol=1e-4, atol=1e-5 * np.abs(H[v]).max())
    # symmetric positive semi-definite blocks; no force or stiffness out of contact
    assert np.allclose(H, np.transpose(H, (0, 2, 1)), atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() >= -1e-12 * np.abs(H).max()
    off = F.lam == 0
    assert np.all(g[off] == 0) and np.all(H[off] == 0)


def test_coulomb_limit_and_stick_spring():
    """Sliding (|u| >= eps_v h): the force has magnitude mu lambda, opposes u,
    and has no normal component.  At rest (u = 0) the force vanishes and the
    stiffness is the spring mu lambda (2 / eps) on the tangent plane."""
    dhat, kappa, h, mu, eps_v = 1e-3, 1e5, 0.01, 0.3, 1e-3
    x_t = np.array([[0.0, 0.0, 5e-4], [1.0, 0.0, 2e-4]])
    F = friction.GroundFriction(mu, eps_v, h, kappa, dhat, [0, 0, 1], 0.0, x_t)
    lam = -kappa * barrier.db(x_t[:, 2], dhat)
    assert np.allclose(F.lam, lam) and np.all(lam > 0)
    x = x_t + np.array([[3e-4, -4e-4, 1e-4], [0.0, 2e-3, 0.0]])    # |u| = 5e-4, 2e-3 > eps = 1e-5
    g = F.gradient(x)
    assert np.allclose(np.linalg.norm(g, axis=1), mu * lam, rtol=1e-14)
    assert np.allclose(g[:, 2], 0, atol=1e-18)
    assert np.all(np.einsum("ij,ij->i", g[:, :2], (x - x_t)[:, :2]) > 0)
    assert np.all(F.gradient(x_t) == 0)
    H0 = F.hessian_blocks(x_t)
    for k in range(2):
        assert np.allclose(H0[k], mu * lam[k] * (2 / F.eps) * np.diag([1.0, 1.0, 0.0]), rtol=1e-14, atol=0)


def test_problem_with_friction_gradient_and_timestep():
    """Eq. IP with the friction term: the gradient is the derivative of E,
    the Hessian is symmetric positive definite, and a timestep of a block
    on the ground with a tangential velocity ends at a minimiser whose
    tangential motion friction has slowed."""
    s = synth.tiny_scene(3, 2, 2, seed=4, contact=True, pinned=False)
    s.x0 = s.x0.copy()
    s.x0[:, 2] += 5e-4 - s.x0[:, 2].min()                       # lowest vertices inside dhat
    s.v0 = np.tile(np.array([0.6, 0.0, 0.0]), (s.n_verts, 1))
    p = ip.Problem(s, mu=0.5, eps_v=1e-3)
    p0 = ip.Problem(s)
    assert p.friction is not None and np.any(p.friction.lam > 0)
    x = p.x_tilde + 1e-4 * rng.normal(size=p.x_tilde.shape)
    x[:, 2] = np.maximum(x[:, 2], 1e-4)
    g = p.gradient(x)
    e = 1e-8
    for v in range(0, s.n_verts, 7):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += e
            xm[v, c] -= e
            fd = (p.energy(xp) - p.energy(xm)) / (2 * e)
            assert fd == pytest.approx(g[v, c], rel=1e-4, abs=1e-7 * np.abs(g).max())
    H = p.hessian(x).toarray()
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0
    x1, info = newton.timestep(p)
    x1_free, _ = newton.timestep(p0)
    assert np.abs(p.gradient(x1)).max() <= 1e-6 * np.abs(p.gradient(p.x_t)).max()
    slide = (x1 - s.x0)[:, 0].mean()
    slide_free = (x1_free - s.x0)[:, 0].mean()
    assert 0 < slide < slide_free
