"""Pins for the oracle's mesh-mesh friction (``friction.PairFriction``, the
lagged IPC friction term D of Eq. IP between bodies), no GPU:

* on a static triangle, a point's friction is the ground friction of the
  plane through the triangle (the pinned point-plane form);
* the gradient and Hessian are the derivatives of D (finite differences),
  the Hessian is PSD and takes its closed form at zero slip;
* motion along the contact normal and common translations carry no
  friction, the forces of a pair sum to zero, and a sliding pair feels the
  Coulomb force mu lambda against its slip;
* in a timestep of two free blocks in contact, total momentum is
  conserved, and a block sliding over the other sticks to it where without
  friction it slides on.
"""
import numpy as np
import pytest

import synth
from oracle import contact, friction, ip, newton

MU, EPS_V, H, KAPPA, DHAT = 0.5, 1e-3, 0.01, 1e3, 0.01
EPS = EPS_V * H


def _apex_over_triangle(d):
    """A large horizontal triangle (the top face of one tet, z = 0) and a
    second tet whose lowest vertex hangs at height d over the triangle's
    interior; only that point-triangle pair is within dhat."""
    X = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0], [0.3, 0.3, -0.5],
                  [0.2, 0.1, d], [1.2, 0.1, 1.0], [0.2, 1.1, 1.0], [0.5, 0.5, 1.3]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    body = np.array([0, 0, 0, 0, 1, 1, 1, 1])
    faces = contact.boundary_faces(tets)
    return X, faces, contact.face_edges(faces), body


DHAT2 = 0.05   # the general configurations: several pairs of every kind within dhat


def _two_tets(seed, gap=0.01):
    """Two tets of different bodies: the upper one's bottom edge (vertices 4
    and 5) lies gap above the lower one's top face z = 0 and crosses the
    face's hypotenuse, vertex 4 over the face's interior and vertex 5 just
    outside it, so that point-triangle pairs with a plane and an edge as
    closest feature and edge-edge pairs with interior and end points as
    closest points all lie within dhat; jittered by the seed."""
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.3, -0.5],
                  [0.2, 0.2, gap], [0.75, 0.32, gap], [0.3, 0.6, 0.6], [0.6, 0.5, 0.8]], dtype=np.float64)
    X[4:, :2] += rng.uniform(-0.01, 0.01, 2)
    X += 1e-3 * rng.normal(size=X.shape)
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    body = np.array([0, 0, 0, 0, 1, 1, 1, 1])
    faces = contact.boundary_faces(tets)
    return X, faces, contact.face_edges(faces), body


def _pf(X, faces, edges, body, dhat=DHAT2):
    return friction.PairFriction(MU, EPS_V, H, KAPPA, dhat, faces, edges, body, X)


@pytest.mark.parametrize("slip", [0.0, 0.3 * EPS, 0.99 * EPS, 3 * EPS, 1e-3])
def test_static_triangle_reduces_to_ground_friction(slip):
    d = 0.004
    X, faces, edges, body = _apex_over_triangle(d)
    pf = _pf(X, faces, edges, body, DHAT)
    assert pf.vids.shape == (1, 4) and pf.n_pt == 1
    gf = friction.GroundFriction(MU, EPS_V, H, KAPPA, DHAT, [0, 0, 1], 0.0, X[4:5])
    rng = np.random.default_rng(1)
    x = X.copy()
    t = rng.normal(size=3)
    x[4] += slip * np.array([t[0], t[1], 0.0]) / np.hypot(t[0], t[1]) + np.array([0, 0, 2e-4])
    assert pf.energy(x) == pytest.approx(gf.energy(x[4:5]), rel=1e-13, abs=1e-300)
    g = pf.gradient(x)
    gg = gf.gradient(x[4:5])[0]
    assert np.allclose(g[4], gg, rtol=1e-12, atol=1e-14 * max(np.abs(gg).max(), 1e-300))
    # the triangle's vertices take the reaction, split by the closest point's weights
    beta = -pf.w[0, 1:]
    assert np.allclose(g[pf.vids[0, 1:]], -beta[:, None] * gg[None], atol=1e-14 * max(np.abs(gg).max(), 1))
    assert not np.any(g[5:])


@pytest.mark.parametrize("seed", [0, 2, 3, 6])   # pairs of all four closest-feature kinds
@pytest.mark.parametrize("scale", [0.3 * EPS, 30 * EPS])
def test_gradient_and_hessian_match_finite_differences(seed, scale):
    X, faces, edges, body = _two_tets(seed)
    pf = _pf(X, faces, edges, body)
    assert len(pf.vids) == 6 and pf.n_pt == 3 and np.all(pf.lam > 0)
    rng = np.random.default_rng(seed + 10)
    x = X + scale * rng.normal(size=X.shape)
    g = pf.gradient(x)
    e = 1e-4 * scale
    for v in range(len(X)):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += e
            xm[v, c] -= e
            fd = (pf.energy(xp) - pf.energy(xm)) / (2 * e)
            assert fd == pytest.approx(g[v, c], rel=1e-5, abs=1e-6 * np.abs(g).max())
    # Hessian of each pair against differences of the gradient, summed into 3n x 3n
    Hs = pf.hessian_pairs(x)
    Hfull = np.zeros((3 * len(X), 3 * len(X)))
    for k, vids in enumerate(pf.vids):
        dof = (3 * vids[:, None] + np.arange(3)[None, :]).ravel()
        Hfull[np.ix_(dof, dof)] += Hs[k]
    for v in range(len(X)):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += e
            xm[v, c] -= e
            col = ((pf.gradient(xp) - pf.gradient(xm)) / (2 * e)).ravel()
            assert np.allclose(Hfull[:, 3 * v + c], col, rtol=1e-4, atol=1e-5 * np.abs(Hfull).max())
    w = np.linalg.eigvalsh(Hs)
    assert w.min() >= -1e-10 * np.abs(w).max()


def test_hessian_at_zero_slip_is_the_closed_form():
    X, faces, edges, body = _two_tets(6)
    pf = _pf(X, faces, edges, body)
    Hs = pf.hessian_pairs(X)
    for k in range(len(pf.vids)):
        Pn = np.eye(3) - np.outer(pf.n[k], pf.n[k])
        ref = np.kron(np.outer(pf.w[k], pf.w[k]), MU * pf.lam[k] * (2.0 / EPS) * Pn)
        assert np.allclose(Hs[k], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_normal_motion_and_common_translation_carry_no_friction():
    X, faces, edges, body = _apex_over_triangle(0.004)
    pf = _pf(X, faces, edges, body, DHAT)
    D0 = pf.energy(X)
    assert D0 == pytest.approx(MU * pf.lam.sum() * EPS / 3.0, rel=1e-14)
    x = X.copy()
    x[4] += 1e-3 * pf.n[0]                               # along the contact normal
    assert pf.energy(x) == pytest.approx(D0, rel=1e-14) and not np.any(pf.gradient(x))
    X2, faces2, edges2, body2 = _two_tets(7)
    pf2 = _pf(X2, faces2, edges2, body2)
    x2 = X2 + np.array([0.01, -0.02, 0.005])             # every vertex by the same vector
    assert pf2.energy(x2) == pytest.approx(pf2.energy(X2), rel=1e-13)
    assert np.abs(pf2.gradient(x2)).max() <= 1e-9 * MU * pf2.lam.max()


@pytest.mark.parametrize("seed", [0, 4])
def test_pair_forces_balance_and_sliding_pairs_feel_coulomb(seed):
    X, faces, edges, body = _two_tets(seed)
    pf = _pf(X, faces, edges, body)
    rng = np.random.default_rng(seed)
    x = X + 50 * EPS * rng.normal(size=X.shape)
    g = pf.gradient(x)
    assert np.abs(g.sum(axis=0)).max() <= 1e-12 * np.abs(g).max()     # forces of every pair sum to zero
    # one sliding pair: its slip |u| >= eps, so the force on its first
    # primitive's closest point is mu lambda against the slip
    pf1 = _pf(X, faces, edges, body)
    k = int(np.argmax(pf1.lam))
    for name in ("vids", "w", "n", "lam"):
        setattr(pf1, name, getattr(pf1, name)[k:k + 1])
    u = pf1._u(x)[0]
    y = np.linalg.norm(u)
    assert y >= EPS
    g1 = pf1.gradient(x)
    w = pf1.w[0]
    f_first = sum(g1[v] for v in pf1.vids[0][:2]) if k >= pf.n_pt else g1[pf1.vids[0][0]]
    share = w[:2].sum() if k >= pf.n_pt else w[0]
    assert np.allclose(f_first, share * MU * pf1.lam[0] * u / y, rtol=1e-12, atol=1e-12 * MU * pf1.lam[0])


def _sliding_blocks(mu):
    """Two free one-voxel blocks 0.5 mm apart (within dhat = 1 mm), the
    upper one sliding sideways at 0.3 m/s, no gravity."""
    s, body = synth.two_block_scene(gap=0.0005, speed=0.0, voxels=(1, 1, 1))
    n0 = int((body == 0).sum())
    s.v0[n0:, 0] = 0.3
    return s, body, n0, ip.Problem(s, body=body, mu=mu, eps_v=EPS_V)


def test_sliding_block_sticks_and_momentum_is_conserved():
    s, body, n0, p = _sliding_blocks(MU)
    assert p.pair_friction is not None and len(p.pair_friction.vids) > 4
    # the gradient of the whole E (friction included) at a trial point
    rng = np.random.default_rng(3)
    x = p.x_tilde + 1e-5 * rng.normal(size=p.x_tilde.shape)
    g = p.gradient(x)
    e = 1e-8
    for v in [n0, n0 + 3, 1, 5]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += e
            xm[v, c] -= e
            fd = (p.energy(xp) - p.energy(xm)) / (2 * e)
            assert fd == pytest.approx(g[v, c], rel=1e-4, abs=1e-6 * np.abs(g).max())
    x1, info = newton.timestep(p)
    assert info["converged"] and p.feasible(x1)
    m = p.mass[:, None]
    p_before = (m * s.v0).sum(axis=0)
    p_after = (m * p.velocity(x1)).sum(axis=0)
    assert np.allclose(p_after, p_before, atol=1e-8 * np.abs(p_before).max())
    # slip at the contacts: each lagged pair's relative tangential
    # displacement over the step (the soft blocks shear, so the bodies' mean
    # displacements differ even where the contacts stick)
    pf = p.pair_friction
    slip = np.linalg.norm(pf._u(x1), axis=1)
    assert slip.max() <= pf.eps                      # every contact sticks
    s0, _, _, p0 = _sliding_blocks(0.0)
    x0, _ = newton.timestep(p0)
    slip0 = np.linalg.norm(pf._u(x0), axis=1)       # without friction: slides on by 0.3 h = 5 mm
    assert np.allclose(slip0, 0.3 * s.dt, rtol=1e-2)


def test_no_pair_within_dhat_gives_no_friction():
    """Bodies farther apart than dhat at x^t: no lagged pair, D = 0, a zero
    gradient, an empty Hessian list, and the problem's H is the frictionless one."""
    s, body = synth.two_block_scene(gap=0.004, speed=0.0, voxels=(1, 1, 1))   # 4 mm > dhat = 1 mm
    n0 = int((body == 0).sum())
    s.v0[n0:, 0] = 0.3
    p = ip.Problem(s, body=body, mu=MU, eps_v=EPS_V)
    pf = p.pair_friction
    assert pf is not None and len(pf.vids) == 0
    x = p.x_tilde
    assert pf.energy(x) == 0.0 and not np.any(pf.gradient(x)) and pf.hessian_pairs(x).shape == (0, 12, 12)
    p0 = ip.Problem(s, body=body)
    assert p.energy(x) == p0.energy(x)
    assert (p.hessian(x) != p0.hessian(x)).nnz == 0
