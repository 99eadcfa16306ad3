"""Projected Newton timestep with filtered backtracking line search (oracle).

The timestep result is x^{t+1} = argmin_x E(x) (Sec. 3.1).  The oracle
reaches it with plain projected Newton: each iteration solves H d = -g
(Eq. 5) exactly, by dense Cholesky, sparse LU or a tight Jacobi-PCG, then
takes a filtered backtracking line search (Sec. 3.9): the initial step is
cut to a fraction of the time of first contact with the ground plane (the
closed-form point-plane CCD), then halved until every tet has J > 0 and the
Armijo condition E(x + a d) <= E(x) + c a g.d holds.  Readings: c = 1e-4,
CCD fraction 0.9, at most 60 halvings.

This stands in for the paper's full-space "IPC-LLT" comparator (Table 2);
the paper's own inexact multilevel direction is a faster route to the same
minimiser and is not reproduced here.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import pcg as opcg

ARMIJO_C = 1e-4
CCD_FRACTION = 0.9
MAX_HALVINGS = 60


def solve_spd(H, rhs, method="auto", rtol=1e-13):
    """Solve H d = rhs for SPD ``H`` (CSR)."""
    n = H.shape[0]
    if method == "auto":
        method = "dense" if n <= 3000 else ("splu" if n <= 120000 else "pcg")
    if method == "dense":
        c = sla.cho_factor(H.toarray(), lower=True)
        return sla.cho_solve(c, rhs)
    if method == "splu":
        return spla.splu(H.tocsc()).solve(rhs)
    if method == "pcg":
        diag = H.diagonal()
        x, info = opcg.pcg(lambda v: H @ v, rhs, lambda r: r / diag, rtol=rtol,
                           max_iter=200000)
        if not info["converged"]:
            raise RuntimeError("oracle PCG did not converge")
        return x
    raise ValueError(method)


def ccd_step_bound(prob, x, d):
    """Largest step fraction allowed by the CCD filter: for the plane,
    min(1, 0.9 * min over approaching vertices of dist_v / (-n . d_v)); with
    bodies, also the mesh-mesh conservative advancement keeping every pair
    at >= 0.1 of its distance (contact.ccd_step)."""
    alpha = 1.0
    if prob.contact:
        dist = prob.distances(x)
        nd = d @ prob.plane_n
        app = nd < 0
        if np.any(app):
            alpha = float(min(1.0, CCD_FRACTION * np.min(dist[app] / (-nd[app]))))
    if getattr(prob, "body", None) is not None:
        from . import contact
        alpha = min(alpha, contact.ccd_step(x, d, prob.faces, prob.edges, prob.body, s=1.0 - CCD_FRACTION))
    return alpha


ROUNDING_REGIME = 1e-13


def _uncut_between_bodies(prob, x, d):
    """True without bodies; with bodies, True when the mesh-mesh CCD filter
    (Sec. 3.9) lets the whole step d through."""
    if getattr(prob, "body", None) is None:
        return True
    from . import contact
    return contact.ccd_step(x, d, prob.faces, prob.edges, prob.body, s=1.0 - CCD_FRACTION) >= 1.0


def line_search(prob, x, d, g, E0):
    """Filtered backtracking.  Returns alpha or raises."""
    alpha = ccd_step_bound(prob, x, d)
    gd = float(np.sum(g * d))
    for _ in range(MAX_HALVINGS + 1):
        xn = x + alpha * d
        if prob.feasible(xn):
            if abs(ARMIJO_C * alpha * gd) <= ROUNDING_REGIME * abs(E0):
                return alpha
            if prob.energy(xn) <= E0 + ARMIJO_C * alpha * gd:
                return alpha
        alpha *= 0.5
    raise RuntimeError("line search failed")


def initial_guess(prob):
    """x_tilde with Dirichlet vertices at x^t; x^t if x_tilde is infeasible.
    With mesh-mesh contact the path from x^t to x_tilde is first cut by the
    CCD filter (a straight move could pass one body through another)."""
    x0 = prob.x_tilde.copy()
    if getattr(prob, "body", None) is not None:
        a = ccd_step_bound(prob, prob.x_t, x0 - prob.x_t)
        x0 = prob.x_t + a * (x0 - prob.x_t)
    if prob.feasible(x0):
        return x0
    return prob.x_t.copy()


def timestep(prob, xtol_rel=1e-12, max_iter=100, method="auto", x_init=None):
    """Minimise E to the step-size tolerance and return (x^{t+1}, info).

    Stops after the first iteration whose Newton direction satisfies
    |d|_inf <= xtol_rel * max(|x - x^t|_inf, h^2 |gravity|); that final
    direction is applied in full when it keeps x feasible and, with bodies,
    when the mesh-mesh CCD filter of Sec. 3.9 does not cut it (a feasible end
    point does not rule out a vertex that passed through a triangle).
    """
    x = initial_guess(prob) if x_init is None else np.array(x_init, dtype=np.float64)
    scale0 = prob.h ** 2 * max(np.linalg.norm(prob.gravity), 1e-30)
    info = {"iters": 0, "gnorm": [], "alpha": [], "converged": False}
    for it in range(max_iter):
        g = prob.gradient(x)
        info["gnorm"].append(float(np.linalg.norm(g)))
        H = prob.hessian(x)
        d = solve_spd(H, -g.ravel(), method=method).reshape(-1, 3)
        d[prob.pinned] = 0.0
        info["iters"] = it + 1
        scale = max(float(np.max(np.abs(x - prob.x_t))), scale0)
        if np.max(np.abs(d)) <= xtol_rel * scale:
            xn = x + d
            if prob.feasible(xn) and _uncut_between_bodies(prob, x, d):
                x = xn
            info["converged"] = True
            break
        E0 = prob.energy(x)
        alpha = line_search(prob, x, d, g, E0)
        info["alpha"].append(alpha)
        x = x + alpha * d
    info["gnorm_final"] = float(np.linalg.norm(prob.gradient(x)))
    return x, info


def paper_timestep(prob, U, n_cg=20, tol=1e-3, max_iter=100):
    """The paper's inexact multilevel timestep (Alg. 1 with Alg. 2's
    directions, Sec. 3.9):

    * each iteration: d_s = U (U^T H U)^{-1} U^T (-g), the subspace levels of
      Alg. 2 solved exactly (with partition-of-unity SMS weights the affine
      space lies inside the SMS space, so the two tight subspace solves give
      this Galerkin direction); d_f = n_cg block-Jacobi CG iterations on
      H d_f = -g - H d_s from zero (Sec. 3.7.2) with the Hessian freshly
      evaluated at the iterate rather than lagged; d = d_s + d_f;
    * the same filtered line search as ``timestep`` (CCD cut, feasibility,
      Armijo);
    * after the update, stop when the mean vertex speed of the subspace
      step, sum_v |d_s,v|_2 / (h n), is below ``tol`` (m/s): the paper's
      test |d_s| / (h |V|) < tol of Sec. 3.9 with |d_s| read per vertex.

    Returns (x^{t+1}, info) with per-iteration step sizes and decrements."""
    from . import subspace
    x = initial_guess(prob)
    info = {"iters": 0, "alpha": [], "decrement": [], "converged": False}
    for it in range(max_iter):
        g = prob.gradient(x)
        g[prob.pinned] = 0.0
        H = prob.hessian(x)
        ds, df = subspace.paper_direction(H, g.ravel(), U, n_cg)
        d = (ds + df).reshape(-1, 3)
        d[prob.pinned] = 0.0
        info["iters"] = it + 1
        gd = float(np.sum(g * d))
        if not gd < 0:
            raise RuntimeError("paper direction is not a descent direction")
        alpha = line_search(prob, x, d, g, prob.energy(x))
        info["alpha"].append(alpha)
        x = x + alpha * d
        dec = float(np.sum(np.linalg.norm(ds.reshape(-1, 3), axis=1)) / (prob.h * prob.n))
        info["decrement"].append(dec)
        if dec < tol:
            info["converged"] = True
            break
    return x, info
