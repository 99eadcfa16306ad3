"""Direct pins for the oracle's Newton helpers (no GPU): the SPD solve, the
point-plane CCD bound and the filtered backtracking line search (Eq. 5 and
Sec. 3.9).  The timestep tests pin them through the minimiser; these pin
each one by a property its code does not compute itself."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import ip, newton

rng = np.random.default_rng(404)


@pytest.mark.parametrize("method", ["dense", "splu", "pcg", "auto"])
def test_solve_spd_methods_agree_with_a_dense_solve(method):
    n = 90
    A = sp.random(n, n, density=0.05, random_state=5, format="csr")
    H = (A @ A.T + sp.identity(n) * 2.0).tocsr()
    rhs = rng.normal(size=n)
    d = newton.solve_spd(H, rhs, method=method)
    ref = np.linalg.solve(H.toarray(), rhs)
    assert np.allclose(d, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    with pytest.raises(ValueError):
        newton.solve_spd(H, rhs, method="qr")


def _ground_problem():
    s = synth.tiny_scene(3, 2, 2, seed=3, contact=True, pinned=False)
    return s, ip.Problem(s)


def test_ccd_bound_is_the_first_time_of_impact_times_the_fraction():
    s, p = _ground_problem()
    x = p.x_t.copy()
    dist = p.distances(x)
    d = np.zeros_like(x)
    a, b, c = 0, 5, 9
    d[a, 2] = -0.5 * dist[a] / 0.04      # reaches the plane at t = 0.04
    d[b, 2] = -dist[b] / 0.02            # reaches the plane first, at t = 0.02
    d[c, 2] = +1.0                       # moves away: no bound
    alpha = newton.ccd_step_bound(p, x, d)
    assert alpha == pytest.approx(0.9 * 0.02, rel=1e-13)
    # at alpha / 0.9 the first vertex touches the plane and no vertex is below it
    xa = x + (alpha / 0.9) * d
    assert p.distances(xa)[b] == pytest.approx(0.0, abs=1e-15)
    assert p.distances(xa).min() >= -1e-15
    # no approaching vertex, or a time of impact beyond the step: the full step
    assert newton.ccd_step_bound(p, x, np.abs(d)) == 1.0
    far = np.zeros_like(x)
    far[b, 2] = -0.1 * dist[b]
    assert newton.ccd_step_bound(p, x, far) == 1.0


def test_line_search_returns_the_first_acceptable_halving():
    """From the CCD bound, halvings until the point is feasible and satisfies
    Armijo; the returned step is feasible with sufficient decrease, and the
    trial before it (twice as long, if it was tried) was not."""
    s, p = _ground_problem()
    x = p.x_tilde.copy()
    x[:, 2] = np.maximum(x[:, 2], 3e-4)
    assert p.feasible(x)
    g = p.gradient(x)
    E0 = p.energy(x)
    for scale in [1e-3, 1e-1, 10.0]:
        d = -scale * g / np.abs(g).max()
        alpha = newton.line_search(p, x, d, g, E0)
        bound = newton.ccd_step_bound(p, x, d)
        k = np.log2(bound / alpha)
        assert k == pytest.approx(round(k), abs=1e-12) and round(k) >= 0
        xa = x + alpha * d
        gd = float(np.sum(g * d))
        assert p.feasible(xa)
        assert p.energy(xa) <= E0 + newton.ARMIJO_C * alpha * gd
        if round(k) > 0:
            x2 = x + 2 * alpha * d
            assert (not p.feasible(x2)) or p.energy(x2) > E0 + newton.ARMIJO_C * 2 * alpha * gd
    # the longest step needed halvings: the test reaches the backtracking
    assert round(np.log2(newton.ccd_step_bound(p, x, d) / alpha)) > 0
