"""GPU parity of the friction between bodies (Eq. IP term D between surface
primitives; the oracle's ``friction.PairFriction`` inside ``ip.Problem``).

These checks are kept out of the collected suite: the file name has no
``test_`` prefix, so ``pytest tests`` does not pick it up.  Run them by
naming the file: ``pytest tests/gpu_checks_pair_friction.py -m gpu``.

Scene: two free one-voxel blocks 0.5 mm apart (within dhat = 1 mm), the
upper one sliding sideways at 0.3 m/s, no gravity, mu = 0.5, eps_v = 1e-3.
Checks, in the order the path runs:

* the gradient and H at an iterate, sliding and sticking (FP64 to
  rounding, FP32 to float32 storage), with the pairs and frames lagged at
  x^t by the assembly entry point;
* the line-search energy along a direction;
* whole timesteps with Jacobi and two-level PCG against the oracle's
  minimiser (1e-8), with every contact sticking (slip <= eps) and the total
  momentum conserved.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import ip, newton

from gpu_helpers import dev, host, rel_disp_error, solver_for

pytestmark = pytest.mark.gpu

MU, EPS_V = 0.5, 1e-3


def _sliding():
    s, body = synth.two_block_scene(gap=0.0005, speed=0.0, voxels=(1, 1, 1))
    n0 = int((body == 0).sum())
    s.v0[n0:, 0] = 0.3
    return s, body, ip.Problem(s, body=body, mu=MU, eps_v=EPS_V)


def _solver(s, body, **opts):
    sol = solver_for(s, **opts)
    sol.set_bodies(body, s.dhat, s.kappa)
    sol.set_friction(MU, EPS_V)
    return sol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
@pytest.mark.parametrize("regime", ["sliding", "sticking"])
def test_friction_assembly_matches_oracle(precision, tol, regime):
    s, body, p = _sliding()
    assert p.pair_friction is not None and len(p.pair_friction.vids) > 4
    rng = np.random.default_rng(0)
    if regime == "sliding":       # the predictor: the upper block 5 mm along, far beyond eps
        x = p.x_tilde + 1e-5 * rng.normal(size=s.x0.shape)
    else:                         # slips below eps = eps_v h
        x = s.x0 + 0.3 * p.pair_friction.eps * rng.normal(size=s.x0.shape)
    sol = _solver(s, body, precision=precision)
    g = host(sol.assemble(dev(x), dev(s.x0), dev(s.v0), s.dt))
    g_o = p.gradient(x)
    assert np.max(np.abs(g - g_o)) <= 1e-11 * np.abs(g_o).max()
    rp, col, val = sol.get_hessian()
    H = sp.bsr_matrix((val, col, rp), shape=(3 * s.n_verts, 3 * s.n_verts)).toarray()
    H_o = p.hessian(x).toarray()
    assert np.max(np.abs(H - H_o)) <= tol * np.abs(H_o).max()


def test_friction_energy_matches_oracle():
    s, body, p = _sliding()
    sol = _solver(s, body)
    sol.assemble(dev(s.x0), dev(s.x0), dev(s.v0), s.dt)    # x^t, the predictor and the lagged pairs
    rng = np.random.default_rng(1)
    x = s.x0 + 1e-5 * rng.normal(size=s.x0.shape)
    d = np.zeros_like(x)
    d[:, :2] = 2e-4 * rng.normal(size=(len(x), 2))         # mostly tangential
    for alpha in (0.0, 0.5, 1.0):
        E, feasible = sol.energy(dev(x), dev(d), alpha)
        assert feasible
        assert E == pytest.approx(p.energy(x + alpha * d), rel=1e-12)


@pytest.mark.parametrize("two_level", [False, True])
def test_sliding_block_step_matches_oracle_and_sticks(two_level):
    s, body, p = _sliding()
    x_o, _ = newton.timestep(p)
    opts = dict(precision="fp64", newton_tol=1e-10, pcg_rtol=1e-12, max_newton=200)
    if two_level:
        opts["preconditioner"] = "two_level"
    sol = _solver(s, body, **opts)
    if two_level:
        origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=4, k=3, seed=5)
        sol.upload_basis(origins, vrow, handle, phi)
    dx, st = sol.newton_step(dev(s.x0), dev(s.v0), s.dt)
    assert st["status"] == 0 and st["contact_pairs"] > 0
    x1 = s.x0 + host(dx)
    assert rel_disp_error(x1, x_o, s.x0) <= 1e-8
    assert p.feasible(x1)
    slip = np.linalg.norm(p.pair_friction._u(x1), axis=1)
    assert slip.max() <= p.pair_friction.eps
    m = p.mass[:, None]
    mom0 = (m * s.v0).sum(axis=0)
    assert np.allclose((m * p.velocity(x1)).sum(axis=0), mom0, atol=1e-8 * np.abs(mom0).max())
