"""Pins for the oracle's barrier, incremental potential, Newton timestep and
PCG (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import barrier, ip, newton, pcg

rng = np.random.default_rng(99)


# -- barrier -----------------------------------------------------------------
def test_barrier_closed_form_points():
    dhat = 1e-3
    # at d = dhat / e: ln(d/dhat) = -1, so b = (d - dhat)^2
    d = dhat / np.e
    assert barrier.b(np.array([d]), dhat)[0] == pytest.approx((d - dhat) ** 2, rel=1e-14)
    assert barrier.db(np.array([d]), dhat)[0] == pytest.approx(2 * (d - dhat) - (d - dhat) ** 2 / d, rel=1e-13)


def test_barrier_vanishes_smoothly_at_dhat():
    dhat = 1e-3
    d = np.array([dhat, 2 * dhat, dhat * (1 - 1e-9)])
    assert np.allclose(barrier.b(d, dhat), 0.0, atol=1e-20)
    assert np.allclose(barrier.db(d, dhat), 0.0, atol=1e-14)
    assert np.allclose(barrier.d2b(d, dhat), 0.0, atol=1e-5)


def test_barrier_derivatives_finite_differences():
    dhat = 1e-3
    d = np.linspace(0.05, 0.95, 19) * dhat
    eps = 1e-10
    fd1 = (barrier.b(d + eps, dhat) - barrier.b(d - eps, dhat)) / (2 * eps)
    fd2 = (barrier.db(d + eps, dhat) - barrier.db(d - eps, dhat)) / (2 * eps)
    assert np.allclose(barrier.db(d, dhat), fd1, rtol=1e-5)
    assert np.allclose(barrier.d2b(d, dhat), fd2, rtol=1e-5)


def test_barrier_convex_and_infinite_below_plane():
    dhat = 1e-3
    d = np.linspace(1e-6, 0.999, 50) * dhat
    assert np.all(barrier.d2b(d, dhat) > 0)
    assert np.isinf(barrier.b(np.array([0.0, -1e-4]), dhat)).all()


# -- incremental potential ----------------------------------------------------
def _problem(contact=False):
    s = synth.tiny_scene(2, 2, 1, seed=7, contact=contact, pinned=not contact)
    return s, ip.Problem(s)


def test_lumped_mass_totals():
    s, p = _problem()
    assert p.mass.sum() == pytest.approx(np.sum(s.rho * p.vol), rel=1e-13)
    # the unit cube's six-tet voxels add up to its volume
    c = ip.Problem(synth.cube_scene())
    assert c.vol.sum() == pytest.approx(1.0, rel=1e-13)
    assert c.mass.sum() == pytest.approx(1000.0, rel=1e-13)


@pytest.mark.parametrize("contact", [False, True])
def test_gradient_matches_finite_differences(contact):
    s, p = _problem(contact)
    x = p.x_tilde + 1e-4 * rng.normal(size=p.x_tilde.shape)
    if contact:
        x[:, 2] = np.maximum(x[:, 2], 2e-4)
    x[p.pinned] = p.x_t[p.pinned]
    g = p.gradient(x)
    eps = 1e-8
    for v in range(0, p.n, 3):
        if p.pinned[v]:
            continue
        for c in range(3):
            xp = x.copy(); xp[v, c] += eps
            xm = x.copy(); xm[v, c] -= eps
            fd = (p.energy(xp) - p.energy(xm)) / (2 * eps)
            assert fd == pytest.approx(g[v, c], rel=1e-4, abs=1e-7 * np.abs(g).max())


@pytest.mark.parametrize("contact", [False, True])
def test_unprojected_hessian_matches_finite_differences(contact):
    s, p = _problem(contact)
    p.project = False
    x = p.x_tilde + 1e-4 * rng.normal(size=p.x_tilde.shape)
    if contact:
        x[:, 2] = np.maximum(x[:, 2], 2e-4)
    x[p.pinned] = p.x_t[p.pinned]
    H = p.hessian(x).toarray()
    eps = 1e-8
    for v in range(p.n):
        if p.pinned[v]:
            continue
        for c in range(3):
            xp = x.copy(); xp[v, c] += eps
            xm = x.copy(); xm[v, c] -= eps
            fd = ((p.gradient(xp) - p.gradient(xm)) / (2 * eps)).ravel()
            col = H[:, 3 * v + c].copy()
            col[np.repeat(p.pinned, 3)] = 0.0
            assert np.allclose(col, fd, rtol=1e-4, atol=1e-6 * np.abs(H).max())


def test_hessian_symmetric_positive_definite():
    s, p = _problem(True)
    x = p.x_tilde.copy()
    H = p.hessian(x).toarray()
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0


@pytest.mark.parametrize("contact", [False, True])
def test_cubature_scaled_hessian_is_affine_in_the_scale(contact):
    """The cubature Hessian (Sec. 3.8) scales only the elastic term:
    unit scales give the full Hessian bit for bit, and since mass and
    barrier terms do not depend on the scale, H(s1) + H(s2) - H(0) =
    H(s1 + s2), and H(s) - H(0) is h^2 times the elastic Hessian weighted by s
    (checked on one element alone, against its own 12 x 12 block)."""
    s, p = _problem(contact)
    x = p.x_tilde + (1e-3 * rng.normal(size=p.x_tilde.shape) if not contact else 0.0)
    x[p.pinned] = p.x_t[p.pinned]
    t = len(s.tets)
    H = p.hessian(x).toarray()
    assert np.array_equal(p.hessian(x, np.ones(t)).toarray(), H)
    s1, s2 = rng.uniform(0, 2, size=t), rng.uniform(0, 2, size=t)
    H0 = p.hessian(x, np.zeros(t)).toarray()
    lhs = p.hessian(x, s1).toarray() + p.hessian(x, s2).toarray() - H0
    assert np.allclose(lhs, p.hessian(x, s1 + s2).toarray(), rtol=0, atol=1e-12 * np.abs(H).max())
    e = int(np.nonzero(~p.pinned[s.tets].any(axis=1))[0][0])   # an element with no pinned vertex
    one = np.zeros(t)
    one[e] = 3.0
    D = p.hessian(x, one).toarray() - H0
    from oracle import elastic
    He = elastic.element_hessian(x, s.tets, p.vol, p.Dm_inv, p.mu, p.lam, project=True)[e]
    dof = (3 * s.tets[e][:, None] + np.arange(3)[None, :]).ravel()
    assert np.allclose(D[np.ix_(dof, dof)], 3.0 * p.h ** 2 * He, rtol=1e-12, atol=1e-12 * np.abs(He).max() * p.h ** 2)
    D[np.ix_(dof, dof)] = 0.0
    assert np.abs(D).max() <= 1e-12 * np.abs(H).max()


def test_bdf2_free_fall_is_exact():
    """BDF2 (Eq. IP with alpha = 4/9, Sec. 3.1) is exact for a quadratic
    trajectory: an undeformed mesh falling freely with exact history
    (x^{t-1}, v^{t-1}) = (x_0, v_0), (x^t, v^t) = (x_0 + v_0 h + g h^2 / 2,
    v_0 + g h) lands on x_0 + 2 v_0 h + 2 g h^2 with v_0 + 2 g h.  Every
    coefficient of the predictor and the velocity update (read from the
    garbled acceleration formula) enters."""
    s = synth.tiny_scene(3, 2, 2, seed=5, pinned=False)
    h = s.dt
    g = np.asarray(s.gravity, dtype=np.float64)
    x0 = s.X + np.array([0.3, -0.2, 1.0])
    v0 = np.tile(np.array([0.5, 0.1, -0.25]), (s.n_verts, 1))
    xt = x0 + v0 * h + 0.5 * g * h * h
    vt = v0 + g * h
    p = ip.Problem(s, x_t=xt, v_t=vt, integrator="bdf2", x_prev=x0, v_prev=v0)
    assert p.alpha == pytest.approx(4.0 / 9.0, rel=0, abs=0)
    x1, info = newton.timestep(p)
    assert np.allclose(x1, x0 + 2 * v0 * h + 2 * g * h * h, rtol=0, atol=1e-12)
    assert np.allclose(p.velocity(x1), v0 + 2 * g * h, rtol=0, atol=1e-10)


def test_bdf2_energy_weights_potentials_by_four_ninths():
    """E = K + (4/9) h^2 (Psi + B) for BDF2 against the same pieces
    computed directly, at a deformed state with contact; the step is a
    minimiser (gradient ~ 0) and its velocity is the BDF2 difference."""
    s = synth.tiny_scene(3, 2, 2, seed=6, contact=True, pinned=False)
    h = s.dt
    rng_l = np.random.default_rng(3)
    xp = s.x0 + 1e-3 * rng_l.normal(size=s.x0.shape)
    vp = 0.1 * rng_l.normal(size=s.x0.shape)
    p = ip.Problem(s, x_t=s.x0, v_t=s.v0, integrator="bdf2", x_prev=xp, v_prev=vp)
    from oracle import elastic
    x = p.x_tilde + 2e-4 * rng_l.normal(size=p.x_tilde.shape)
    x[:, 2] = np.maximum(x[:, 2], 2e-4)
    K = 0.5 * np.sum(p.mass[:, None] * (x - p.x_tilde) ** 2)
    Psi = np.sum(elastic.element_energy(x, s.tets, p.vol, p.Dm_inv, p.mu, p.lam))
    B = p.kappa * np.sum(barrier.b(p.distances(x), p.dhat))
    assert p.energy(x) == pytest.approx(K + (4.0 / 9.0) * h * h * (Psi + B), rel=1e-13)
    x1, info = newton.timestep(p)
    assert np.abs(p.gradient(x1)).max() <= 1e-6 * np.abs(p.gradient(p.x_t)).max()
    assert np.allclose(p.velocity(x1), (3 * x1 - 4 * s.x0 + xp) / (2 * h), rtol=1e-14, atol=0)


def test_bdf2_is_implicit_euler_of_two_thirds_step():
    """The reading the GPU's BDF2 step rests on: Eq. IP with alpha = 4/9 is
    the implicit-Euler potential of the step h' = 2h/3 around the BDF2
    predictor.  An implicit-Euler problem with h' and the velocity v' that
    puts its predictor x^t + h' v' + h'^2 g on the BDF2 one has the same E,
    gradient, Hessian and minimiser, friction included (its mollifier width
    eps_v h' matched by eps_v' = 3 eps_v / 2).  A wrong alpha, predictor
    coefficient or width breaks the equality."""
    s = synth.tiny_scene(3, 2, 2, seed=7, contact=True, pinned=False)
    h = s.dt
    g = np.asarray(s.gravity, dtype=np.float64)
    rng_l = np.random.default_rng(4)
    s.v0 = np.tile(np.array([0.4, -0.1, 0.0]), (s.n_verts, 1)) + 0.05 * rng_l.normal(size=s.x0.shape)
    xp = s.x0 - h * s.v0 + 1e-4 * rng_l.normal(size=s.x0.shape)
    vp = s.v0 + 0.05 * rng_l.normal(size=s.x0.shape)
    pb = ip.Problem(s, integrator="bdf2", x_prev=xp, v_prev=vp, mu=0.4, eps_v=1e-3)
    h2 = 2.0 * h / 3.0
    v_eq = (pb.x_tilde - s.x0 - h2 * h2 * g[None, :]) / h2
    pe = ip.Problem(s, v_t=v_eq, dt=h2, mu=0.4, eps_v=1.5e-3)
    assert np.allclose(pe.x_tilde, pb.x_tilde, rtol=0, atol=1e-15)
    assert pe.ah2 == pytest.approx(pb.ah2, rel=1e-15)
    x = pb.x_tilde + 3e-4 * rng_l.normal(size=s.x0.shape)
    # every other vertex inside the mollifier (slip < eps = 1.7e-5), where D depends on its width
    x[::2] = s.x0[::2] + 3e-6 * rng_l.normal(size=s.x0[::2].shape)
    x[:, 2] = np.maximum(x[:, 2], 2e-4)
    assert pe.energy(x) == pytest.approx(pb.energy(x), rel=1e-13)
    gb = pb.gradient(x)
    assert np.allclose(pe.gradient(x), gb, rtol=0, atol=1e-12 * np.abs(gb).max())
    Hb = pb.hessian(x).toarray()
    assert np.allclose(pe.hessian(x).toarray(), Hb, rtol=0, atol=1e-12 * np.abs(Hb).max())
    xb, _ = newton.timestep(pb)
    xe, _ = newton.timestep(pe)
    assert np.linalg.norm(xe - xb) <= 1e-9 * np.linalg.norm(xb - s.x0)


# -- Newton timestep -----------------------------------------------------------
def test_uniform_translation_is_exact():
    """No gravity, no contact, no pins: a rigid translation with velocity v
    costs no elastic energy, so x^{t+1} = x^t + h v exactly."""
    s = synth.tiny_scene(2, 2, 2, seed=1, pinned=False)
    s.gravity = (0.0, 0.0, 0.0)
    v = np.array([0.3, -1.2, 0.7])
    s.v0 = np.broadcast_to(v, s.X.shape).copy()
    p = ip.Problem(s)
    x, info = newton.timestep(p)
    assert np.allclose(x, s.x0 + s.dt * v[None, :], atol=1e-14)


def test_rest_without_forces_stays():
    s = synth.tiny_scene(2, 1, 1, seed=2, pinned=True)
    s.gravity = (0.0, 0.0, 0.0)
    s.v0 = np.zeros_like(s.X)
    x, info = newton.timestep(ip.Problem(s))
    assert np.abs(x - s.x0).max() <= 1e-15


@pytest.mark.parametrize("contact", [False, True])
def test_timestep_is_a_minimiser(contact):
    """KKT by finite differences of E (independent of the analytic gradient),
    and every feasible perturbation raises E."""
    s = synth.tiny_scene(2, 2, 1, seed=11, contact=contact, pinned=not contact)
    p = ip.Problem(s)
    x, info = newton.timestep(p)
    assert info["converged"]
    E0 = p.energy(x)
    scale = np.abs(x - p.x_t).max()
    for trial in range(10):
        dv = rng.normal(size=x.shape)
        dv[p.pinned] = 0
        dv *= 1e-3 * scale / np.abs(dv).max()
        assert p.energy(x + dv) > E0
        assert p.energy(x - dv) > E0
    g = p.gradient(x)
    assert np.linalg.norm(g) <= 1e-9 * np.linalg.norm(p.mass[:, None] * (x - p.x_tilde)) + 1e-14


def test_minimiser_unique_from_two_starts():
    s = synth.tiny_scene(3, 2, 1, seed=4, contact=True, pinned=False)
    p = ip.Problem(s)
    xa, _ = newton.timestep(p)
    xb, _ = newton.timestep(p, x_init=p.x_t)
    assert np.abs(xa - xb).max() <= 1e-12 * np.abs(xa - p.x_t).max()


def test_cube_newton_reaches_grad_norm():
    s = synth.cube_scene()
    p = ip.Problem(s)
    x, info = newton.timestep(p)
    assert info["converged"] and info["gnorm_final"] <= 1e-8
    # the dense direct solve and the sparse LU give the same minimiser
    x2, _ = newton.timestep(p, method="splu")
    assert np.abs(x - x2).max() <= 1e-12 * np.abs(x - p.x_t).max()


def test_contact_keeps_vertices_above_plane():
    s = synth.tiny_scene(3, 2, 2, seed=8, contact=True, pinned=False)
    s.v0[:] = np.array([0.0, 0.0, -2.0])
    p = ip.Problem(s)
    x, info = newton.timestep(p)
    assert p.distances(x).min() > 0
    # with the barrier switched off the same step would cross the plane
    assert (p.x_tilde[:, 2]).min() < 0


# -- PCG -------------------------------------------------------------------------
def test_pcg_solves_random_spd():
    n = 40
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)
    b = rng.normal(size=n)
    x, info = pcg.pcg(lambda v: A @ v, b, lambda r: r / np.diag(A), rtol=1e-12)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_pcg_exact_preconditioner_one_iteration():
    n = 30
    A = rng.normal(size=(n, n))
    A = A @ A.T + np.eye(n)
    b = rng.normal(size=n)
    Ainv = np.linalg.inv(A)
    x, info = pcg.pcg(lambda v: A @ v, b, lambda r: Ainv @ r, rtol=1e-10)
    assert info["iters"] == 1


def test_paper_timestep_limits():
    """The paper's inexact timestep: with a basis spanning every free degree
    of freedom the subspace direction is the Newton direction, so with a
    vanishing tolerance it reaches the exact timestep's minimiser; with a
    small basis and the paper's settings (20 CG iterations, 1e-3 m/s) it
    stops on its decrement, lowers the energy, and its result is close to
    (but not at) the minimiser."""
    import scipy.sparse as sp
    from oracle import subspace
    s = synth.tiny_scene(4, 2, 2, seed=12, E_range=(1e5, 1e7))
    p = ip.Problem(s)
    x_o, _ = newton.timestep(p)
    full = sp.csr_matrix(np.eye(3 * s.n_verts))
    x1, info = newton.paper_timestep(p, full, n_cg=0, tol=1e-13)
    assert info["converged"]
    assert np.linalg.norm(x1 - x_o) <= 1e-9 * np.linalg.norm(x_o - s.x0)
    o, vr, h, ph = synth.random_sparse_basis(s.X, m=4, k=2, seed=1)
    U = subspace.lbs_basis_matrix(s.X, o, vr, h, ph)
    x2, info2 = newton.paper_timestep(p, U, n_cg=20, tol=1e-3)
    assert info2["converged"] and info2["decrement"][-1] < 1e-3
    assert p.energy(x2) < p.energy(newton.initial_guess(p))
    err = np.linalg.norm(x2 - x_o) / np.linalg.norm(x_o - s.x0)
    assert 0 < err < 0.5
