"""Parity on the named workloads, in the configuration the benchmark runs.

* Beam (40x10x10 voxels, 24,000 tets, E in {1e5, 1e9}, clamped end): one
  timestep against the oracle's converged minimiser -- FP64 paths within
  1e-9 and the mixed-precision two-level path within 1e-4 per-step relative
  displacement, using the paper's SMS basis (32 handles).
* Full-size lattice (41^3, 224,226 tets, ground contact): the oracle cannot
  converge a full-size timestep in seconds, so the check is (a) per-tet
  parity of element energies, gradients and projected Hessians on a sample
  of tets at a deformed contact state, and (b) the oracle's Newton correction
  at the GPU's result, e = H^{-1} g with the oracle's Hessian and gradient
  (solved by the oracle's Jacobi-PCG to 1e-3 relative residual), as the
  displacement error estimate |e| / |x^{t+1} - x^t| against the same
  1e-9 / 1e-4 bars.
"""
import numpy as np
import pytest

import synth
from oracle import elastic, ip, newton, pcg

from gpu_helpers import dev, host, rel_disp_error, solver_for, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def beam():
    s = synth.beam_scene()
    p = ip.Problem(s)
    x_o, info = newton.timestep(p, method="splu")
    from paper_2508_13386_gb300 import basis
    B = basis.build_sms_basis(s.X, s.tets, s.E, 32, dirichlet=s.dirichlet, seed=1)
    return s, p, x_o, B


@pytest.mark.parametrize("precision,precond,tol", [
    ("fp64", "jacobi", 1e-9),
    ("fp64", "two_level", 1e-9),
    ("fp32", "two_level", 1e-4),
])
def test_beam_timestep(beam, precision, precond, tol):
    s, p, x_o, B = beam
    solver = solver_for(s, precision=precision, preconditioner=precond,
                        newton_tol=1e-10 if precision == "fp64" else 1e-6)
    if precond == "two_level":
        solver.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    dx, stats = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    err = rel_disp_error(s.x0 + host(dx), x_o, s.x0)
    assert err <= tol, (err, stats)


def test_beam_timestep_with_cubature_coarse_operator(beam):
    """The SMS basis with its modal moment-fitting cubature (Sec. 3.8, Alg.
    3) building the coarse operator: the preconditioner changes, the
    timestep does not (it matches the oracle's), and the cubature keeps a
    small fraction of the elements."""
    from paper_2508_13386_gb300 import cubature
    s, p, x_o, B = beam
    C = cubature.build_cubature(s.X, s.tets, B, seed=0, workers=1)
    assert len(C["elem"]) < len(s.tets) // 4
    solver = solver_for(s, precision="fp64", preconditioner="two_level", newton_tol=1e-10)
    solver.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    solver.upload_cubature(C["scale"])
    dx, stats = solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert rel_disp_error(s.x0 + host(dx), x_o, s.x0) <= 1e-9, stats


def test_beam_bf16_reports_indefinite_operator(beam):
    """bfloat16 keeps 8 mantissa bits: with E = 1e9 next to E = 1e5 the
    rounded H is indefinite (its rounding error exceeds the mass term in the
    stiff blocks' rigid modes).  The coarse operator, summed in float64 from
    the stored H, still factors, and PCG meets the non-positive curvature:
    the library reports MLS_ENONFINITE (-7, a PCG breakdown) instead of
    returning a wrong step."""
    import paper_2508_13386_gb300 as mls
    s, p, x_o, B = beam
    solver = solver_for(s, precision="bf16", preconditioner="two_level", newton_tol=1e-6)
    solver.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    with pytest.raises(mls.MLSError) as e:
        solver.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert e.value.status == -7 and "PCG breakdown" in str(e.value)


def test_beam_two_level_cuts_pcg_iterations(beam):
    s, p, x_o, B = beam
    jac = solver_for(s, precision="fp64", preconditioner="jacobi")
    _, st_j = jac.newton_step(dev(s.x0), dev(s.v0), s.dt)
    ml = solver_for(s, precision="fp64", preconditioner="two_level")
    ml.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    _, st_m = ml.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert st_m["pcg_iters"] < 0.5 * st_j["pcg_iters"]


def _deformed_beam_state(s, p, U, amplitude, seed):
    """x_tilde plus a random coarse displacement U q (Dirichlet rows of U are
    zero), halved until every tet keeps a positive volume."""
    rng = np.random.default_rng(seed)
    q = rng.normal(size=U.shape[1])
    d = (U @ q).reshape(-1, 3)
    d *= amplitude / np.abs(d).max()
    for _ in range(30):
        x = p.x_tilde + d
        if np.isfinite(p.energy(x)):
            return x
        d *= 0.5
    raise AssertionError("no feasible deformed state")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_stiff_beam_coarse_operator_is_spd_and_matches_oracle(beam, precision):
    """U^T H U of the 1e5/1e9 Pa beam at a strongly deformed state (the
    warm-start kind of iterate x_tilde + U q, a few centimetres of coarse
    motion): its smallest eigenvalues are differences of terms ~1e4x larger
    (near-rigid motions of stiff cells, whose elastic parts cancel down to
    the mass), so the library sums it in float64 from H's stored values.
    Element by element it matches the oracle's dense triple product U^T H U
    (Alg. 2), it is positive definite and spectrally equivalent to the
    oracle's operator (the generalized eigenvalues of (A, A_oracle) near 1),
    and the factorisation needs no diagonal shift.  In float64 the entries
    agree to 1e-10 of sqrt(A_ii A_jj); in float32 H itself is stored rounded,
    so the entries agree to 1e-5 of the largest, as in the Galerkin parity
    test, and the spectrum within a factor of two."""
    from oracle import subspace
    s, p, x_o, B = beam
    U = subspace.lbs_basis_matrix(s.X, B["origins"], B["vrow"], B["handle"], B["phi"])
    x = _deformed_beam_state(s, p, U, 0.03, seed=11)
    solver = solver_for(s, precision=precision, preconditioner="two_level")
    solver.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    solver.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt)
    solver.build_coarse()
    A = solver.get_coarse()
    A_o = subspace.galerkin(p.hessian(x), U)
    A_o = A_o.toarray() if hasattr(A_o, "toarray") else np.asarray(A_o)
    import scipy.linalg as sla
    if precision == "fp64":
        d = np.sqrt(np.abs(np.diag(A_o)))
        assert np.max(np.abs(A - A_o) / np.outer(d, d)) <= 1e-10
    else:
        assert np.max(np.abs(A - A_o)) <= 1e-5 * np.abs(A_o).max()
    np.linalg.cholesky(A)
    lam = sla.eigh(A, A_o, eigvals_only=True)
    band = 1e-8 if precision == "fp64" else 0.5
    assert lam[0] >= 1 - band and lam[-1] <= 1 + (band if precision == "fp64" else 1.0), (lam[0], lam[-1])
    assert solver.coarse_shift() == 0.0


@pytest.fixture(scope="module")
def lattice_state():
    """The full-size lattice after three steps of the benchmark trajectory."""
    from paper_2508_13386_gb300 import basis
    s = synth.lattice_scene(n=41, seed=3, v_down=1.0)
    B = basis.build_sms_basis(s.X, s.tets, s.E, 160, seed=1)
    solver = solver_for(s, precision="fp32", preconditioner="two_level", newton_tol=1e-5, coarse_refresh=1)
    solver.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    x = dev(s.x0)
    v = dev(s.v0)
    for _ in range(3):
        dx, st = solver.newton_step(x, v, s.dt)
        v.copy_(dx / s.dt)
        x.add_(dx)
    return s, B, host(x), host(v)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_fullsize_element_parity_sampled(lattice_state, precision, rtol):
    s, B, x, v = lattice_state
    solver = solver_for(s, precision=precision)
    E, g, H = solver.eval_elements(dev(x))
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(s.n_tets, size=3000, replace=False))
    tets = s.tets[idx]
    vol, Dm_inv = elastic.rest_shape(s.X, tets)
    mu, lam = elastic.lame(s.E[idx], s.nu[idx])
    E_o = elastic.element_energy(x, tets, vol, Dm_inv, mu, lam)
    g_o = elastic.element_gradient(x, tets, vol, Dm_inv, mu, lam)
    H_o = elastic.element_hessian(x, tets, vol, Dm_inv, mu, lam, project=True)
    # psi ~ strain^2 is a difference of O(strain) terms, so near-rigid tets
    # lose relative accuracy in any FP64 evaluation order: compare on the
    # element's own scale vol (mu + lam)
    escale = vol * (mu + lam)
    assert np.all(np.abs(host(E)[idx] - E_o) <= 1e-12 * escale + 1e-10 * np.abs(E_o))
    # P = mu (F - F^-T) + lam ln J F^-T also cancels at small strain: compare on
    # the element's unit-strain force scale vol (mu + lam) |Dm^-1|
    fscale = (vol * (mu + lam) * np.abs(Dm_inv).max(axis=(1, 2)))[:, None]
    assert np.all(np.abs(host(g)[idx] - g_o) <= 1e-13 * fscale + 1e-10 * np.abs(g_o))
    Hs = np.abs(H_o).max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(host(H)[idx] - H_o) / Hs) <= rtol


BENCH_SETTINGS = dict(newton_tol=1e-3, pcg_rtol=1e-2, coarse_refresh=1000, coarse_lag_steps=7, omega=0.0,
                      cycle="multiplicative", pcg_check_every=8)


@pytest.mark.parametrize("precision,precond,tol,settings", [
    ("fp64", "jacobi", 1e-9, dict(newton_tol=1e-10, coarse_refresh=1)),
    ("fp32", "two_level", 1e-4, dict(newton_tol=1e-6, coarse_refresh=1)),
    ("fp32", "two_level", 1e-4, BENCH_SETTINGS),   # the benchmark's timed settings
])
def test_fullsize_timestep_gradient_bound(lattice_state, precision, precond, tol, settings):
    s, B, x, v = lattice_state
    p = ip.Problem(s, x_t=x, v_t=v, threads=8)
    solver = solver_for(s, precision=precision, preconditioner=precond, **settings)
    if precond == "two_level":
        solver.upload_basis(B["origins"], B["vrow"], B["handle"], B["phi"])
    dx, stats = solver.newton_step(dev(x), dev(v), s.dt)
    x1 = x + host(dx)
    assert p.feasible(x1)
    g = p.gradient(x1).ravel()
    H = p.hessian(x1)
    diag = H.diagonal()
    e, info = pcg.pcg(lambda u: H @ u, g, lambda r: r / diag, rtol=1e-3, max_iter=5000)
    est = np.linalg.norm(e) / np.linalg.norm(x1 - x)
    assert est <= tol, (est, stats)
