"""What a learned PCG initial guess in the coarse space can gain, on the
oracle (no GPU).

The learned warm start predicts the coarse coordinates of the step.  Used as
the initial guess d0 = U c of a Newton system H d = b, the best any predictor
can do is the Galerkin projection of the exact solution d*:
c* = (U^T H U)^{-1} U^T H d*.  Because H d* = b, that is
c* = (U^T H U)^{-1} U^T b: the coarse solve of the right-hand side (the
deflation initial guess), which needs no predictor at all.  These tests pin
that identity, and measure, with the oracle's two-level PCG (the
multiplicative cycle of Alg. 2's preconditioner with an exact coarse solve),
what that ideal guess saves on the stiff beam (1e5 / 1e9 Pa cells) dropped
from rest:

* on the first Newton system of the step, whose solution is almost all
  coarse (the ideal guess leaves under 2% of its H-norm), the solve to the
  relative residual 1e-2 needs at most 2 iterations instead of 7;
* on the second, where the ideal guess leaves about half of the H-norm, it
  saves at most 2 of about 15 iterations;
* on the third, whose solution is almost all fine-scale (over 99% left), it
  saves at most one of several hundred.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import ip, newton, pcg, subspace


@pytest.fixture(scope="module")
def beam_systems():
    s = synth.beam_scene()
    p = ip.Problem(s)
    origins, vrow, handle, phi = synth.random_sparse_basis(s.X, m=8, k=3, seed=1)
    U = sp.diags(np.repeat(~p.pinned, 3).astype(np.float64)) @ \
        subspace.lbs_basis_matrix(s.X, origins, vrow, handle, phi)
    x = newton.initial_guess(p)
    systems = []
    for it in range(3):
        g = p.gradient(x)
        H = p.hessian(x).tocsc()
        b = -g.ravel()
        dstar = spla.splu(H).solve(b)
        systems.append((H, b, dstar))
        alpha = newton.line_search(p, x, dstar.reshape(-1, 3), g, p.energy(x))
        x = x + alpha * dstar.reshape(-1, 3)
    return U, systems


def _iters(H, U, b, x0, rtol=1e-2):
    Ac = subspace.galerkin(H, U)
    Dinv = subspace.block_diagonal_inverse(H)
    M = lambda r: subspace.two_level_apply(H, U, Ac, r, mode="multiplicative", omega=0.6, Dinv=Dinv)
    _, info = pcg.pcg(lambda v: H @ v, b, M, rtol=rtol, x0=x0)
    assert info["converged"]
    return info["iters"]


def test_ideal_coarse_guess_is_the_coarse_solve_of_the_right_hand_side(beam_systems):
    U, systems = beam_systems
    H, b, dstar = systems[0]
    Ac = subspace.galerkin(H, U)
    c_proj = subspace.coarse_solve(Ac, U.T @ (H @ dstar))
    c_rhs = subspace.coarse_solve(Ac, U.T @ b)
    assert np.allclose(c_proj, c_rhs, rtol=1e-8, atol=1e-8 * np.abs(c_rhs).max())
    # and it is the best coarse guess in the H-norm: any perturbation of c is worse
    e = lambda c: (dstar - U @ c) @ (H @ (dstar - U @ c))
    rng = np.random.default_rng(0)
    for _ in range(5):
        assert e(c_rhs + 1e-3 * np.abs(c_rhs).max() * rng.normal(size=c_rhs.shape)) > e(c_rhs)


def test_ideal_coarse_guess_helps_only_a_mostly_coarse_system(beam_systems):
    U, systems = beam_systems
    saved = []
    for k, (H, b, dstar) in enumerate(systems):
        Ac = subspace.galerkin(H, U)
        d0 = U @ subspace.coarse_solve(Ac, U.T @ b)
        left = np.sqrt((dstar - d0) @ (H @ (dstar - d0)) / (dstar @ (H @ dstar)))
        i0, i1 = _iters(H, U, b, None), _iters(H, U, b, d0)
        saved.append(i0 - i1)
        if k == 0:
            assert left < 0.02 and i0 >= 5 and i1 <= 2
        elif k == 1:
            assert 0.3 < left < 0.8 and i0 - i1 <= 2
        else:
            assert left > 0.99 and i0 >= 100 and i0 - i1 <= 1
