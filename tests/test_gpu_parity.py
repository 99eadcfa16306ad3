"""Parity of each row of the hot path: CUDA kernels (through the C ABI) vs
the FP64 oracle on the same seeded inputs.

Tolerances: float64 kernels agree with the oracle to rounding (relative 1e-10
on element quantities, 1e-9 on the timestep result); float32 kernels to
1e-4 relative on element Hessians (FP32 eigen-decomposition of a 3x3 with
condition up to ~1e3) and the mixed-precision timestep to 1e-4 per-step
relative displacement, the stated target for the mixed path.
"""
import numpy as np
import pytest

import synth
from oracle import elastic, ip, newton, subspace

from gpu_helpers import dev, host, rel_disp_error, solver_for, torch

pytestmark = pytest.mark.gpu

rng = np.random.default_rng(2024)


def _deformed(scene, amp=0.02, compress=None):
    x = scene.X + amp * rng.normal(size=scene.X.shape) * 0.1
    if compress is not None:
        x = x * np.asarray(compress)[None, :]
    return x


# ---- S2: element energy / gradient / projected Hessian ------------------------------------
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 2e-4)])
@pytest.mark.parametrize("compress", [None, (0.7, 1.0, 1.1), (1.3, 0.8, 0.9)])
def test_element_eval_matches_oracle(precision, rtol, compress):
    s = synth.tiny_scene(4, 3, 2, seed=31)
    x = _deformed(s, compress=compress)
    solver = solver_for(s, precision=precision)
    E, g, H = solver.eval_elements(dev(x))
    vol, Dm_inv = elastic.rest_shape(s.X, s.tets)
    mu, lam = elastic.lame(s.E, s.nu)
    E_o = elastic.element_energy(x, s.tets, vol, Dm_inv, mu, lam)
    g_o = elastic.element_gradient(x, s.tets, vol, Dm_inv, mu, lam)
    H_o = elastic.element_hessian(x, s.tets, vol, Dm_inv, mu, lam, project=True)
    assert np.allclose(host(E), E_o, rtol=1e-12, atol=1e-12 * np.abs(E_o).max())
    assert np.allclose(host(g), g_o, rtol=1e-11, atol=1e-11 * np.abs(g_o).max())
    Hg = host(H)
    scale = np.abs(H_o).max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(Hg - H_o) / scale) <= rtol


def test_element_eval_inverted_tet_is_infinite():
    s = synth.tiny_scene(1, 1, 1, seed=2)
    x = s.X.copy()
    x[:, 0] *= -1.0  # mirror: every tet inverted
    E, g, H = solver_for(s).eval_elements(dev(x))
    assert np.all(np.isinf(host(E)))


# ---- S4/S5: gradient and BSR assembly --------------------------------------------------------
@pytest.mark.parametrize("contact", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_assembly_matches_oracle(contact, precision):
    s = synth.tiny_scene(5, 3, 3, seed=8, contact=contact, pinned=not contact)
    p = ip.Problem(s)
    x = p.x_tilde + 2e-4 * rng.normal(size=p.x_tilde.shape)
    if contact:
        x[:, 2] = np.maximum(x[:, 2], 1e-4)
    x[p.pinned] = p.x_t[p.pinned]
    solver = solver_for(s, precision=precision)
    g = host(solver.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt))
    g_o = p.gradient(x)
    assert np.allclose(g, g_o, rtol=1e-11, atol=1e-11 * np.abs(g_o).max())
    rp, col, val = solver.get_hessian()
    import scipy.sparse as sp
    H = sp.bsr_matrix((val, col, rp), shape=(3 * s.n_verts, 3 * s.n_verts)).toarray()
    H_o = p.hessian(x).toarray()
    tol = {"fp64": 1e-11, "fp32": 2e-5, "bf16": 1e-2}[precision]
    assert np.max(np.abs(H - H_o)) <= tol * np.abs(H_o).max()
    # the block pattern is the vertex adjacency through tets
    assert len(col) == len({(int(a), int(b)) for t in s.tets for a in t for b in t})


# ---- S8: SpMV and PCG ---------------------------------------------------------------------
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_spmv_matches_oracle(precision, tol):
    s = synth.tiny_scene(7, 4, 3, seed=3)   # several 32-row slices, ragged tail
    p = ip.Problem(s)
    solver = solver_for(s, precision=precision)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    v = rng.normal(size=s.X.shape)
    y = host(solver.spmv(dev(v)))
    H = p.hessian(p.x_tilde)
    y_o = (H @ v.ravel()).reshape(-1, 3)
    assert np.max(np.abs(y - y_o)) <= tol * np.abs(H).max() * np.abs(v).max() * 16


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_pcg_solves_newton_system(precision, rtol, persistent):
    s = synth.tiny_scene(6, 3, 3, seed=5, E_range=(1e5, 1e8))
    p = ip.Problem(s)
    solver = solver_for(s, precision=precision, persistent=persistent)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    H = p.hessian(p.x_tilde)
    b = -p.gradient(p.x_tilde)
    d, iters, rel, st = solver.pcg_solve(dev(b), rtol=rtol, max_iter=5000)
    d_o = newton.solve_spd(H, b.ravel(), method="dense").reshape(-1, 3)
    r_true = np.linalg.norm(b.ravel() - H @ host(d).ravel()) / np.linalg.norm(b)
    assert st == 0 and iters > 0
    assert r_true <= 10 * rtol
    # error bound through the condition number of H
    cond = np.linalg.cond(H.toarray())
    assert np.linalg.norm(host(d) - d_o) <= 10 * rtol * cond * np.linalg.norm(d_o)


@pytest.mark.parametrize("cycle", ["additive", "multiplicative"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_two_level_pcg_matches_phase_kernels(precision, cycle):
    """The persistent PCG kernel and the one-launch-per-phase loop run the
    same iteration (only the order of the float64 reductions differs): same
    iteration count within one, same solution to the solve tolerance, and
    the true residual of both within the tolerance."""
    s = synth.tiny_scene(9, 4, 3, seed=21, E_range=(1e5, 1e9))   # 200 vertices: 7 slices, ragged tail
    p = ip.Problem(s)
    H = p.hessian(p.x_tilde)
    b = -p.gradient(p.x_tilde)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=2)
    rtol = 1e-9 if precision == "fp64" else 1e-5
    out = []
    for persistent in (True, False):
        solver = solver_for(s, precision=precision, preconditioner="two_level", cycle=cycle, omega=0.5,
                            persistent=persistent)
        solver.upload_basis(origins, vrow, handle, phi)
        solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
        solver.build_coarse()
        d, iters, rel, st = solver.pcg_solve(dev(b), rtol=rtol, max_iter=2000)
        assert st == 0 and iters > 0
        dh = host(d)
        assert np.linalg.norm(b.ravel() - H @ dh.ravel()) <= 10 * rtol * np.linalg.norm(b)
        out.append((dh, iters))
    (d1, i1), (d2, i2) = out
    assert abs(i1 - i2) <= 1
    if i1 == i2:   # same iteration: only reduction rounding separates the iterates
        assert np.linalg.norm(d1 - d2) <= (rtol if precision == "fp64" else 1e-4) * np.linalg.norm(d2)


@pytest.mark.parametrize("precond", ["jacobi", "two_level"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pcg_repeats_bitwise_and_stops_at_the_cap(precision, precond):
    """The dot products of the PCG loop are summed as integers in fixed
    point, so the order in which blocks add them does not matter: the same
    solve twice gives the same bits and the same count.  A cap below the
    converged count stops with MLS_ENOTCONV after exactly that many
    iterations, inside a host check chunk (16 iterations) and at its ends."""
    s = synth.tiny_scene(9, 4, 3, seed=21, E_range=(1e5, 1e9))
    p = ip.Problem(s)
    H = p.hessian(p.x_tilde)
    b = -p.gradient(p.x_tilde)
    solver = solver_for(s, precision=precision, preconditioner=precond, cycle="multiplicative", omega=0.5)
    if precond == "two_level":
        origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=2)
        solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    if precond == "two_level":
        solver.build_coarse()
    rtol = 1e-9 if precision == "fp64" else 1e-5
    d1, i1, r1, st1 = solver.pcg_solve(dev(b), rtol=rtol, max_iter=5000)
    d2, i2, r2, st2 = solver.pcg_solve(dev(b), rtol=rtol, max_iter=5000)
    assert st1 == 0 and st2 == 0 and i1 == i2 and r1 == r2
    assert np.array_equal(host(d1), host(d2))
    assert np.linalg.norm(b.ravel() - H @ host(d1).ravel()) <= 10 * rtol * np.linalg.norm(b)
    for cap in (1, 7, 15, 16, 17, 32):
        if cap < i1:
            d, it, rel, st = solver.pcg_solve(dev(b), rtol=rtol, max_iter=cap)
            assert st == -4 and it == cap, (cap, it, st)
            assert rel > rtol


@pytest.mark.parametrize("precond", ["jacobi", "two_level"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pcg_fixed_point_sums_follow_the_scale(precision, precond):
    """The fixed-point PCG sums take their scale from the previous value of
    each dot product.  Scaling the right-hand side by 2^k scales every dot
    product by 2^2k and nothing else: the solve takes the same iterations and
    returns the scaled solution bit for bit (powers of two are exact).
    k = +-80 for float64 vectors; k = +-40 for float vectors, which keeps
    their smallest entries normal."""
    s = synth.tiny_scene(9, 4, 3, seed=21, E_range=(1e5, 1e9))
    p = ip.Problem(s)
    b = -p.gradient(p.x_tilde)
    solver = solver_for(s, precision=precision, preconditioner=precond, cycle="multiplicative", omega=0.5)
    if precond == "two_level":
        origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=2)
        solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    if precond == "two_level":
        solver.build_coarse()
    rtol = 1e-9 if precision == "fp64" else 1e-5
    d0, i0, r0, st0 = solver.pcg_solve(dev(b), rtol=rtol, max_iter=5000)
    assert st0 == 0
    k = 80 if precision == "fp64" else 40
    for scale in (2.0 ** k, 2.0 ** -k):
        d, i, r, st = solver.pcg_solve(dev(b * scale), rtol=rtol, max_iter=5000)
        assert st == 0 and i == i0
        assert np.array_equal(host(d), host(d0) * scale)


def test_pcg_zero_rhs():
    s = synth.tiny_scene(2, 2, 2, seed=1)
    p = ip.Problem(s)
    solver = solver_for(s)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    d, iters, rel, st = solver.pcg_solve(dev(np.zeros_like(s.X)), rtol=1e-8)
    assert iters == 0 and np.all(host(d) == 0)


# ---- S9: energy, feasibility, CCD -------------------------------------------------------------
def test_energy_and_ccd_match_oracle():
    s = synth.tiny_scene(4, 3, 2, seed=9, contact=True, pinned=False)
    s.v0[:] = np.array([0.0, 0.0, -1.0])
    p = ip.Problem(s)
    solver = solver_for(s)
    x = p.x_t.copy()
    solver.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt)
    d = p.x_tilde - x
    for alpha in [0.0, 0.1, 0.3]:
        E, feas = solver.energy(dev(x), dev(d), alpha)
        xa = x + alpha * d
        assert feas == p.feasible(xa)
        if feas:
            assert E == pytest.approx(p.energy(xa), rel=1e-12)
    a = solver.ccd_bound(dev(x), dev(d))
    assert a == pytest.approx(newton.ccd_step_bound(p, x, d), rel=1e-14)
    E, feas = solver.energy(dev(x), dev(d), 1.0)
    assert not feas and not p.feasible(x + d)


# ---- S1-S10: the full timestep --------------------------------------------------------------
def _step(scene, **opts):
    solver = solver_for(scene, **opts)
    x = dev(scene.x0)
    v = dev(scene.v0)
    dx, stats = solver.newton_step(x, v, scene.dt)
    return scene.x0 + host(dx), stats


def test_cube_timestep_fp64():
    s = synth.cube_scene()
    p = ip.Problem(s)
    x_o, info = newton.timestep(p)
    x_g, stats = _step(s, precision="fp64")
    assert rel_disp_error(x_g, x_o, s.x0) <= 1e-9
    assert np.linalg.norm(p.gradient(x_g)) <= 1e-8   # the cube's stated Newton tolerance
    assert stats["newton_iters"] <= 20


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 1e-4)])
def test_cube_timestep_mixed(precision, tol):
    s = synth.cube_scene()
    p = ip.Problem(s)
    x_o, _ = newton.timestep(p)
    x_g, stats = _step(s, precision=precision, newton_tol=1e-6)
    assert rel_disp_error(x_g, x_o, s.x0) <= tol


def test_contact_timestep_fp64():
    s = synth.tiny_scene(4, 3, 2, seed=12, contact=True, pinned=False)
    s.v0[:] = np.array([0.2, 0.0, -1.5])
    p = ip.Problem(s)
    x_o, info = newton.timestep(p)
    x_g, stats = _step(s, precision="fp64")
    assert p.distances(x_g).min() > 0
    assert rel_disp_error(x_g, x_o, s.x0) <= 1e-9


def test_translation_exact_on_gpu():
    s = synth.tiny_scene(3, 2, 2, seed=1, pinned=False)
    s.gravity = (0.0, 0.0, 0.0)
    vel = np.array([0.3, -1.2, 0.7])
    s.v0 = np.broadcast_to(vel, s.X.shape).copy()
    x_g, _ = _step(s)
    assert np.allclose(x_g, s.x0 + s.dt * vel[None, :], atol=1e-14)


def test_host_entry_point_matches_device_entry_point():
    s = synth.tiny_scene(3, 3, 2, seed=6)
    solver = solver_for(s)
    dx_d, _ = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    dx_h, _ = solver.newton_step_host(s.x0, s.v0, s.dt)
    assert np.array_equal(host(dx_d), dx_h)


# ---- basis kernels (S5/S6 of the two-level path) ----------------------------------------------
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_prolong_restrict_match_oracle(precision, tol):
    s = synth.tiny_scene(6, 4, 3, seed=14)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=9, k=4, seed=2)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    solver = solver_for(s, precision=precision)
    solver.upload_basis(origins, vrow, handle, phi)
    q = rng.normal(size=(9, 12))
    w = host(solver.prolong(dev(q)))
    w_o = subspace.prolong(U, q)
    assert np.max(np.abs(w - w_o)) <= tol * 10 * np.abs(w_o).max()
    r = rng.normal(size=s.X.shape)
    z = host(solver.restrict(dev(r)))
    z_o = subspace.restrict(U, r)
    assert np.max(np.abs(z - z_o)) <= tol * 100 * np.abs(z_o).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_galerkin_matches_oracle(precision, tol):
    s = synth.tiny_scene(6, 4, 3, seed=15, E_range=(1e5, 1e8))
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=3)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    solver = solver_for(s, precision=precision, preconditioner="two_level")
    solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    A = solver.get_coarse()
    A_o = subspace.galerkin(p.hessian(p.x_tilde), U)
    assert np.max(np.abs(A - A_o)) <= tol * np.abs(A_o).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("contact", [False, True])
def test_cubature_galerkin_matches_oracle(precision, tol, contact):
    """With a cubature of the elastic term (Sec. 3.8) the coarse operator is
    U^T H_cub U, H_cub = M + h^2 (sum_e s_e H_e + barrier): random factors,
    half of them zero, against the oracle's scaled Hessian; the fine H stays
    the full one, and removing the cubature restores the full operator."""
    s = synth.tiny_scene(6, 4, 3, seed=15, E_range=(1e5, 1e8), contact=contact, pinned=not contact)
    p = ip.Problem(s)
    x = p.x_tilde.copy()
    if contact:
        x[:, 2] = np.maximum(x[:, 2], 2e-4)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=3)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    t = len(s.tets)
    cub = rng.uniform(0.0, 2.0, size=t) * (rng.random(t) < 0.5)
    solver = solver_for(s, precision=precision, preconditioner="two_level")
    solver.upload_basis(origins, vrow, handle, phi)
    solver.upload_cubature(cub)
    solver.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    A = solver.get_coarse()
    A_o = subspace.galerkin(p.hessian(x, cub), U)
    assert np.max(np.abs(A - A_o)) <= tol * np.abs(A_o).max()
    import scipy.sparse as sp
    rp, col, val = solver.get_hessian()
    H = sp.bsr_matrix((val, col, rp), shape=(3 * s.n_verts, 3 * s.n_verts)).toarray()
    H_o = p.hessian(x).toarray()
    assert np.max(np.abs(H - H_o)) <= {"fp64": 1e-11, "fp32": 2e-5}[precision] * np.abs(H_o).max()
    solver.upload_cubature(None)
    solver.build_coarse()
    A_full = subspace.galerkin(p.hessian(x), U)
    assert np.max(np.abs(solver.get_coarse() - A_full)) <= tol * np.abs(A_full).max()


@pytest.mark.parametrize("cycle", ["additive", "multiplicative"])
def test_two_level_apply_matches_oracle(cycle):
    s = synth.tiny_scene(6, 4, 3, seed=16, E_range=(1e5, 1e8), pinned=False)
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=4)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    solver = solver_for(s, precision="fp64", preconditioner="two_level", cycle=cycle, omega=0.5)
    solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    H = p.hessian(p.x_tilde)
    r = rng.normal(size=s.X.shape)
    z = host(solver.precond_apply(dev(r)))
    z_o = subspace.two_level_apply(H, U, subspace.galerkin(H, U), r.ravel(), mode=cycle,
                                   omega=0.5).reshape(-1, 3)
    assert np.max(np.abs(z - z_o)) <= 1e-8 * np.abs(z_o).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 2e-3)])
def test_two_level_apply_many_coarse_tiles(precision, tol):
    """A 516 x 516 coarse operator (16 full 32 x 32 tiles of the blocked
    Cholesky and a ragged 4-row one; condition number ~2e4 from E in
    [1e5, 1e9]; four 128-wide panels, whose trailing updates run on the
    tensor cores in sliced bf16 products): the preconditioner apply through
    the factor and its inverse matches the oracle's dense solve."""
    s = synth.tiny_scene(12, 8, 6, seed=18, E_range=(1e5, 1e9), pinned=False)
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=43, k=4, seed=6)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    solver = solver_for(s, precision=precision, preconditioner="two_level", cycle="multiplicative", omega=0.5)
    solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    H = p.hessian(p.x_tilde)
    r = rng.normal(size=s.X.shape)
    z = host(solver.precond_apply(dev(r)))
    z_o = subspace.two_level_apply(H, U, subspace.galerkin(H, U), r.ravel(), mode="multiplicative",
                                   omega=0.5).reshape(-1, 3)
    assert np.max(np.abs(z - z_o)) <= tol * np.abs(z_o).max()


def test_tensor_core_coarse_factor_float64_accuracy():
    """A 1,320 x 1,320 coarse operator (110 handles; 42 tiles of 32, ten
    128-wide panels whose rank-128 trailing updates are exact sums of bf16
    slice products on the tensor cores, E in [1e5, 1e9]): the factor's
    backward error is below 1e-14 r, and the FP64 two-level apply, which
    solves with the factor and its inverse, matches the oracle's dense solve
    to 1e-9, as a float64 factorisation must."""
    s = synth.tiny_scene(16, 12, 8, seed=23, E_range=(1e5, 1e9), pinned=False)
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=110, k=4, seed=9)
    U = subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    solver = solver_for(s, precision="fp64", preconditioner="two_level", cycle="multiplicative", omega=0.5)
    solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    assert solver.coarse_shift() == 0.0
    # the factor itself: backward error ||L L^T - A|| / ||A|| <= 1e-14 r
    A = solver.get_coarse()
    L = solver.get_coarse_factor()
    r = A.shape[0]
    assert np.linalg.norm(L @ L.T - A) <= 1e-14 * r * np.linalg.norm(A)
    H = p.hessian(p.x_tilde)
    Ac = subspace.galerkin(H, U)
    for seed in range(2):
        r = np.random.default_rng(100 + seed).normal(size=s.X.shape)
        z = host(solver.precond_apply(dev(r)))
        z_o = subspace.two_level_apply(H, U, Ac, r.ravel(), mode="multiplicative", omega=0.5).reshape(-1, 3)
        assert np.max(np.abs(z - z_o)) <= 1e-9 * np.abs(z_o).max()


def test_singular_coarse_operator_reported():
    """A handle that no vertex uses makes U^T H U singular (12 zero rows):
    the factorisation meets a zero pivot and the library reports
    MLS_ECHOL (-6) instead of returning a factor."""
    import paper_2508_13386_gb300 as mls
    s = synth.tiny_scene(6, 4, 3, seed=19)
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=7)
    origins = np.vstack([origins, s.X.mean(axis=0)])  # handle 7: no vertices
    solver = solver_for(s, precision="fp64", preconditioner="two_level")
    solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    with pytest.raises(mls.MLSError) as e:
        solver.build_coarse()
    assert e.value.status == -6


def test_indefinite_coarse_operator_falls_back_to_block_jacobi():
    """A timestep whose coarse operator stays singular after every
    diagonal-shift retry (a handle with no vertices: 12 zero rows, which a
    relative diagonal shift cannot lift) preconditions each Newton iteration
    with block Jacobi instead of failing; the stats count the four shifted
    retries and the fallback of every iteration, and the step still matches
    the oracle's minimiser."""
    s = synth.tiny_scene(6, 4, 3, seed=19)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=7, k=3, seed=7)
    origins = np.vstack([origins, s.X.mean(axis=0)])  # handle 7: no vertices
    solver = solver_for(s, precision="fp64", preconditioner="two_level", newton_tol=1e-10)
    solver.upload_basis(origins, vrow, handle, phi)
    dx, st = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    x_o, _ = newton.timestep(ip.Problem(s))
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-9
    assert st["coarse_fallbacks"] >= 1 and st["coarse_builds"] == 0
    assert st["coarse_shifts"] == 4 * st["coarse_fallbacks"]


def test_lagged_coarse_factor_keeps_the_timestep():
    """coarse_lag_steps = 2: a step's first Newton iteration reuses a coarse
    factor built at most two steps earlier, so over four steps the factor is
    built on steps 0 and 3 only.  The lagged factor only preconditions: each
    step still matches the oracle's timestep from the same state."""
    s = synth.tiny_scene(8, 3, 3, seed=21, E_range=(1e5, 1e9))
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=6, k=3, seed=5)
    solver = solver_for(s, precision="fp64", preconditioner="two_level", newton_tol=1e-10,
                        coarse_refresh=1000, coarse_lag_steps=2)
    solver.upload_basis(origins, vrow, handle, phi)
    x, v = s.x0.copy(), s.v0.copy()
    builds = []
    for _ in range(4):
        dx, st = solver.newton_step(dev(x), dev(v), s.dt)
        builds.append(st["coarse_builds"])
        x_o, _ = newton.timestep(ip.Problem(s, x_t=x, v_t=v))
        x_new = x + host(dx)
        assert rel_disp_error(x_new, x_o, x) <= 1e-9
        v = (x_new - x) / s.dt
        x = x_new
    assert builds == [1, 0, 0, 1]


def test_automatic_smoother_damping_tracks_lambda_max():
    """omega = 0: at the coarse build the library estimates lambda_max(D^-1 H)
    (D the 3x3 block diagonal) by 20 Lanczos steps and damps the smoother
    with omega = 0.9 x 2 / lambda.  The estimate matches the largest
    generalized eigenvalue of (H, D) from the oracle's Hessian, never exceeds
    it, and a timestep with that damping matches the oracle's timestep."""
    import scipy.linalg as sla
    s = synth.tiny_scene(8, 3, 3, seed=17, E_range=(1e5, 1e9))
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=6, k=3, seed=5)
    solver = solver_for(s, precision="fp64", preconditioner="two_level", cycle="multiplicative", omega=0.0,
                        newton_tol=1e-10)
    solver.upload_basis(origins, vrow, handle, phi)
    solver.assemble(dev(p.x_tilde), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    omega, lam = solver.smoother_omega()
    H = p.hessian(p.x_tilde).toarray()
    D = np.zeros_like(H)
    for v in range(s.n_verts):
        D[3 * v:3 * v + 3, 3 * v:3 * v + 3] = H[3 * v:3 * v + 3, 3 * v:3 * v + 3]
    lam_o = sla.eigh(H, D, eigvals_only=True).max()
    assert lam_o * (1 - 1e-3) <= lam <= lam_o * (1 + 1e-9), (lam, lam_o)
    assert omega == pytest.approx(1.8 / lam, rel=1e-12)
    x_o, _ = newton.timestep(p)
    dx, st = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-9


def test_two_level_timestep_fp64_beam_slice():
    s = synth.tiny_scene(8, 3, 3, seed=17, E_range=(1e5, 1e9))
    p = ip.Problem(s)
    x_o, _ = newton.timestep(p)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=6, k=3, seed=5)
    solver = solver_for(s, precision="fp64", preconditioner="two_level")
    solver.upload_basis(origins, vrow, handle, phi)
    dx, stats = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-9


# ---- boundary errors ----------------------------------------------------------------------------
def test_invalid_inputs_rejected():
    import paper_2508_13386_gb300 as mls
    s = synth.tiny_scene(2, 1, 1, seed=1)
    solver = mls.Solver()
    bad = s.tets.copy()
    bad[0, 0] = s.n_verts  # out of range
    with pytest.raises(mls.MLSError, match="EINVAL"):
        solver.upload_mesh(s.X, bad, s.E, s.nu, s.rho)
    with pytest.raises(mls.MLSError, match="EINVAL"):
        solver.upload_mesh(s.X[:0], s.tets[:0], s.E[:0], s.nu[:0], s.rho[:0])
    flipped = s.tets[:, [1, 0, 2, 3]]
    with pytest.raises(mls.MLSError, match="EINVAL"):
        solver.upload_mesh(s.X, flipped, s.E, s.nu, s.rho)
    solver.setup_scene(s)
    x = s.X.copy()
    x[:, 0] *= -1.0
    with pytest.raises(mls.MLSError, match="EINVERTED"):
        solver.newton_step(dev(x), dev(s.v0), s.dt)


# ---- bounded device waits ---------------------------------------------------------------------
def test_bounded_barrier_wait_gives_up_and_context_survives():
    """The grid barrier of the persistent PCG kernel bounds its wait: with
    one arrival more than there are blocks nothing releases it, every block
    gives up after its poll limit and the call reports MLS_ETIMEOUT; with
    the right count it releases.  The context stays usable afterwards."""
    import ctypes as C
    import paper_2508_13386_gb300 as mls
    lib = mls._get_lib()
    gave = C.c_int32(-1)
    assert lib.mls_selftest_barrier(8, 9, 20000, C.byref(gave), None) == -8
    assert gave.value == 8
    assert lib.mls_selftest_barrier(8, 8, 20000, C.byref(gave), None) == 0
    assert gave.value == 0
    s = synth.tiny_scene(3, 2, 2, seed=4)
    x_o, _ = newton.timestep(ip.Problem(s))
    solver = solver_for(s, precision="fp64")
    dx, st = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-9
