"""Lagged point-plane friction and the BDF2 timestep on the GPU, against the
FP64 oracle (Eq. IP with the friction term D; Sec. 3.1's BDF2 integrator).

The GPU path adds D's gradient, diagonal Hessian blocks and energy in the
assembly and line-search kernels, and runs BDF2 as the implicit-Euler
potential of the step 2h/3 around the BDF2 predictor.  Tolerances are those
of the other timestep parity tests: float64 assembly to 1e-11 of the largest
entry, line-search energies to 1e-12 relative, float64 timesteps to 1e-9
per-step relative displacement, float32 ones to 1e-4.
"""
import numpy as np
import pytest

import synth
from oracle import ip, newton

from gpu_helpers import dev, host, rel_disp_error, solver_for

pytestmark = pytest.mark.gpu

MU = 0.5
EPS_V = 1e-3


def _ground_block(speed, seed=4):
    """A 3x2x2-voxel block whose lowest vertices sit inside dhat of the ground,
    moving along +x at ``speed`` m/s (no pins, gravity on)."""
    s = synth.tiny_scene(3, 2, 2, seed=seed, contact=True, pinned=False)
    s.x0 = s.x0.copy()
    s.x0[:, 2] += 5e-4 - s.x0[:, 2].min()
    s.v0 = np.tile(np.array([speed, 0.0, 0.0]), (s.n_verts, 1))
    return s


def _friction_solver(scene, **opts):
    solver = solver_for(scene, **opts)
    solver.set_friction(MU, EPS_V)
    return solver


# ---- friction terms of the assembly and the line-search energy --------------------------
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
@pytest.mark.parametrize("slip", [1e-7, 3e-5, 1e-3])
def test_friction_gradient_and_hessian_match_oracle(precision, tol, slip):
    """slip sets the tangential displacement against the mollifier width
    eps = eps_v h = 1.7e-5 m: sticking, inside the mollifier, sliding."""
    rng = np.random.default_rng(31)
    s = synth.tiny_scene(5, 3, 3, seed=8, contact=True, pinned=False)
    p = ip.Problem(s, mu=MU, eps_v=EPS_V)
    assert np.any(p.friction.lam > 0) and np.any(p.friction.lam == 0)
    x = p.x_t + slip * rng.normal(size=p.x_t.shape)
    x[:, 2] = np.maximum(p.x_t[:, 2] + 1e-5 * rng.normal(size=s.n_verts), 1e-4)
    solver = _friction_solver(s, precision=precision)
    g = host(solver.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt))
    g_o = p.gradient(x)
    assert np.allclose(g, g_o, rtol=1e-11, atol=1e-11 * np.abs(g_o).max())
    rp, col, val = solver.get_hessian()
    import scipy.sparse as sp
    H = sp.bsr_matrix((val, col, rp), shape=(3 * s.n_verts, 3 * s.n_verts)).toarray()
    H_o = p.hessian(x).toarray()
    assert np.max(np.abs(H - H_o)) <= tol * np.abs(H_o).max()
    # the case has friction stiffness to check: without it the diagonal differs
    H_plain = ip.Problem(s).hessian(x).toarray()
    assert np.max(np.abs(H_o - H_plain)) > 1e-6 * np.abs(H_o).max()


def test_friction_energy_matches_oracle():
    rng = np.random.default_rng(32)
    s = _ground_block(0.6)
    p = ip.Problem(s, mu=MU, eps_v=EPS_V)
    solver = _friction_solver(s)
    x = p.x_t.copy()
    solver.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt)
    d = p.x_tilde - x + 1e-4 * rng.normal(size=x.shape)
    d[:, 2] = np.abs(d[:, 2])
    for alpha in [0.0, 1e-3, 0.1, 1.0]:
        E, feas = solver.energy(dev(x), dev(d), alpha)
        xa = x + alpha * d
        assert feas == p.feasible(xa)
        assert E == pytest.approx(p.energy(xa), rel=1e-12)


# ---- implicit-Euler timestep with friction ---------------------------------------------
@pytest.mark.parametrize("speed", [0.6, 1e-4])
def test_friction_timestep_matches_oracle(speed):
    """Sliding (0.6 m/s: 1 cm per step, far beyond eps) and sticking
    (1e-4 m/s: inside the mollifier) blocks on the ground."""
    s = _ground_block(speed)
    p = ip.Problem(s, mu=MU, eps_v=EPS_V)
    x_o, _ = newton.timestep(p)
    solver = _friction_solver(s, precision="fp64")
    dx, stats = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    x_g = s.x0 + host(dx)
    assert p.distances(x_g).min() > 0
    assert rel_disp_error(x_g, x_o, s.x0) <= 1e-9
    if speed > 0.1:
        # friction slows the slide against the same step without it
        plain = solver_for(s, precision="fp64")
        dx0, _ = plain.newton_step(dev(s.x0), dev(s.v0), s.dt)
        slide, slide_free = host(dx)[:, 0].mean(), host(dx0)[:, 0].mean()
        assert 0 < slide < slide_free


def test_friction_off_and_invalid_settings():
    s = _ground_block(0.6)
    solver = solver_for(s)
    import paper_2508_13386_gb300 as mls
    with pytest.raises(mls.MLSError):
        solver.set_friction(-0.1)
    with pytest.raises(mls.MLSError):
        solver.set_friction(0.3, 0.0)
    solver.set_forces(s.gravity, False)
    with pytest.raises(mls.MLSError):
        solver.set_friction(0.3)
    # mu = 0 is the plain step, bit for bit
    a = solver_for(s)
    b = solver_for(s)
    b.set_friction(0.0)
    dxa, _ = a.newton_step(dev(s.x0), dev(s.v0), s.dt)
    dxb, _ = b.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert np.array_equal(host(dxa), host(dxb))


# ---- BDF2 ---------------------------------------------------------------------------------
def test_bdf2_free_fall_is_exact():
    """A rigid, unstrained block in free fall: the BDF2 minimiser is the
    predictor itself (the elastic energy vanishes on translations)."""
    s = synth.tiny_scene(3, 2, 2, seed=1, pinned=False)
    h = s.dt
    g = np.asarray(s.gravity, dtype=np.float64)
    v_prev = np.broadcast_to(np.array([0.3, -0.2, 0.1]), s.X.shape).copy()
    v_t = v_prev + h * g[None, :]
    x_prev = s.X + np.array([0.01, 0.02, 0.3])
    x_t = x_prev + h * v_t
    x_tilde = (4 * x_t - x_prev) / 3 + (2 * h / 9) * (4 * v_t - v_prev) + (4 * h * h / 9) * g[None, :]
    solver = solver_for(s)
    dx, stats = solver.newton_step_bdf2(dev(x_t), dev(v_t), dev(x_prev), dev(v_prev), h)
    assert np.allclose(host(dx), x_tilde - x_t, rtol=0, atol=1e-14)
    assert stats["newton_iters"] <= 2


@pytest.mark.parametrize("precision,tol,newton_tol", [("fp64", 1e-9, 1e-10), ("fp32", 1e-4, 1e-6)])
def test_bdf2_timestep_matches_oracle(precision, tol, newton_tol):
    """Second step of the pinned cube: an implicit-Euler first step (oracle)
    gives the history, then one BDF2 step from it on both sides."""
    s = synth.cube_scene()
    h = s.dt
    x1, _ = newton.timestep(ip.Problem(s))
    v1 = (x1 - s.x0) / h
    p = ip.Problem(s, x_t=x1, v_t=v1, integrator="bdf2", x_prev=s.x0, v_prev=s.v0)
    x2, _ = newton.timestep(p)
    solver = solver_for(s, precision=precision, newton_tol=newton_tol)
    dx, stats = solver.newton_step_bdf2(dev(x1), dev(v1), dev(s.x0), dev(s.v0), h)
    x2_g = x1 + host(dx)
    assert rel_disp_error(x2_g, x2, x1) <= tol


def test_bdf2_with_friction_matches_oracle():
    s = _ground_block(0.6, seed=5)
    h = s.dt
    x_prev = s.x0 - h * s.v0
    v_prev = s.v0.copy()
    p = ip.Problem(s, integrator="bdf2", x_prev=x_prev, v_prev=v_prev, mu=MU, eps_v=EPS_V)
    x_o, _ = newton.timestep(p)
    solver = _friction_solver(s, precision="fp64")
    dx, _ = solver.newton_step_bdf2(dev(s.x0), dev(s.v0), dev(x_prev), dev(v_prev), h)
    x_g = s.x0 + host(dx)
    assert p.distances(x_g).min() > 0
    assert rel_disp_error(x_g, x_o, s.x0) <= 1e-9


# ---- the batched path --------------------------------------------------------------------
def test_batch_with_friction_matches_oracle_per_mesh():
    """Friction on every mesh of a batch (one graph launch per step): each
    mesh against the oracle's friction timestep from the same state."""
    import paper_2508_13386_gb300 as mls
    scenes = [_ground_block(0.6, seed=4), _ground_block(1e-4, seed=5),
              synth.tiny_scene(5, 3, 2, seed=2, contact=True, pinned=False, E_range=(1e5, 1e9))]
    b = mls.Batch(precision="fp64", newton_tol=1e-10)
    b.upload_scenes(scenes)
    b.set_friction(MU, EPS_V)
    x = dev(np.concatenate([s.x0 for s in scenes]))
    v = dev(np.concatenate([s.v0 for s in scenes]))
    dx, stats, info = b.step(x, v, scenes[0].dt)
    assert info["status"] == 0
    dxh = host(dx)
    k = 0
    for sc, st in zip(scenes, stats):
        sl = slice(k, k + sc.n_verts)
        k += sc.n_verts
        assert st["status"] == 0
        x_o, _ = newton.timestep(ip.Problem(sc, mu=MU, eps_v=EPS_V))
        assert rel_disp_error(sc.x0 + dxh[sl], x_o, sc.x0) <= 1e-9


def test_batch_bdf2_with_friction_matches_oracle_and_switches_back():
    """BDF2 steps of a batch with friction, each mesh against the oracle's
    BDF2 step; then an implicit-Euler step on the same batch (the step graph
    is rebuilt for each integrator) against the oracle's implicit Euler."""
    import paper_2508_13386_gb300 as mls
    scenes = [_ground_block(0.6, seed=4), synth.tiny_scene(4, 3, 2, seed=6, contact=True, pinned=True)]
    h = scenes[0].dt
    b = mls.Batch(precision="fp64", newton_tol=1e-10)
    b.upload_scenes(scenes)
    b.set_friction(MU, EPS_V)
    x_prev = [s.x0 - h * s.v0 for s in scenes]
    for sc, xp in zip(scenes, x_prev):
        xp[np.asarray(sc.dirichlet, bool)] = sc.x0[np.asarray(sc.dirichlet, bool)]
    cat = lambda arrs: dev(np.concatenate(arrs))            # noqa: E731
    x, v = cat([s.x0 for s in scenes]), cat([s.v0 for s in scenes])
    dx, stats, info = b.step_bdf2(x, v, cat(x_prev), cat([s.v0 for s in scenes]), h)
    assert info["status"] == 0
    dx_ie, stats_ie, info_ie = b.step(x, v, h)
    assert info_ie["status"] == 0
    dxh, dxh_ie = host(dx), host(dx_ie)
    k = 0
    for sc, xp, st in zip(scenes, x_prev, stats):
        sl = slice(k, k + sc.n_verts)
        k += sc.n_verts
        assert st["status"] == 0
        p = ip.Problem(sc, integrator="bdf2", x_prev=xp, v_prev=sc.v0, mu=MU, eps_v=EPS_V)
        x_o, _ = newton.timestep(p)
        assert rel_disp_error(sc.x0 + dxh[sl], x_o, sc.x0) <= 1e-9
        x_ie, _ = newton.timestep(ip.Problem(sc, mu=MU, eps_v=EPS_V))
        assert rel_disp_error(sc.x0 + dxh_ie[sl], x_ie, sc.x0) <= 1e-9
