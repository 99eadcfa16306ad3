"""Pins for the oracle's mesh-mesh contact primitives (no GPU): closest
distances against dense sampling and closed forms, the barrier gradient
against finite differences, and the conservative CCD against exact times of
impact."""
import numpy as np
import pytest

from oracle import contact

rng = np.random.default_rng(21)


def _tri_samples(a, b, c, k=120):
    u, v = np.meshgrid(np.linspace(0, 1, k), np.linspace(0, 1, k))
    m = (u + v) <= 1
    u, v = u[m], v[m]
    return a[None] + u[:, None] * (b - a)[None] + v[:, None] * (c - a)[None]


def test_point_triangle_distance_against_sampling():
    for _ in range(60):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 1.5
        d = contact.point_triangle_distance(p, a, b, c)
        S = _tri_samples(a, b, c)
        ds = np.linalg.norm(S - p, axis=1).min()
        assert d <= ds + 1e-12                      # no sample is closer
        h = max(np.linalg.norm(b - a), np.linalg.norm(c - a)) / 119
        assert ds - d <= 2 * h                      # and the sampling gets within its spacing


def test_point_triangle_closed_forms():
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    assert contact.point_triangle_distance([0.2, 0.3, 0.7], a, b, c) == pytest.approx(0.7, abs=1e-15)
    assert contact.point_triangle_distance([-1.0, -1.0, 0.0], a, b, c) == pytest.approx(np.sqrt(2), abs=1e-15)
    assert contact.point_triangle_distance([1.0, 1.0, 0.0], a, b, c) == pytest.approx(np.sqrt(0.5), abs=1e-15)
    assert contact.point_triangle_distance([0.5, -2.0, 1.0], a, b, c) == pytest.approx(np.sqrt(5), abs=1e-15)


def test_edge_edge_distance_against_sampling_and_closed_forms():
    t = np.linspace(0, 1, 401)
    for _ in range(60):
        p0, p1, q0, q1 = rng.normal(size=(4, 3))
        d = contact.edge_edge_distance(p0, p1, q0, q1)
        P = p0[None] + t[:, None] * (p1 - p0)[None]
        Q = q0[None] + t[:, None] * (q1 - q0)[None]
        ds = np.linalg.norm(P[:, None] - Q[None], axis=2).min()
        assert d <= ds + 1e-12
        assert ds - d <= (np.linalg.norm(p1 - p0) + np.linalg.norm(q1 - q0)) / 400
    # skew and perpendicular, offset 0.5; parallel, separation 0.3; crossing
    assert contact.edge_edge_distance([0, 0, 0], [1, 0, 0], [0.5, -1, 0.5], [0.5, 1, 0.5]) == pytest.approx(0.5)
    assert contact.edge_edge_distance([0, 0, 0], [1, 0, 0], [0.2, 0.3, 0], [2.0, 0.3, 0]) == pytest.approx(0.3)
    assert contact.edge_edge_distance([0, 0, 0], [1, 0, 0], [0.5, -1, 0], [0.5, 1, 0]) == pytest.approx(0.0, abs=1e-15)
    # segments whose lines meet outside both: endpoint to endpoint
    assert contact.edge_edge_distance([0, 0, 0], [1, 0, 0], [2, 1, 0], [2, 3, 0]) == pytest.approx(np.sqrt(2))


def test_boundary_faces_of_one_tet_and_two_glued_tets():
    assert len(contact.boundary_faces(np.array([[0, 1, 2, 3]]))) == 4
    f = contact.boundary_faces(np.array([[0, 1, 2, 3], [1, 2, 3, 4]]))
    assert len(f) == 6 and not any(set(r) == {1, 2, 3} for r in f.tolist())
    assert len(contact.face_edges(f)) == 9


def _two_tets(gap):
    """Two separate tets (bodies 0 and 1), the second above the first with a
    vertex pointing down at the first's top face; ``gap`` between them."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.3, -0.5],
                  [0.3, 0.3, 0], [1.3, 0.3, 0.6], [0.3, 1.3, 0.6], [0.6, 0.6, 0.9]], dtype=np.float64)
    X[4:, 2] += gap
    X[4:, :2] += np.array([0.02, -0.01])
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    body = np.array([0, 0, 0, 0, 1, 1, 1, 1])
    return X, tets, body


def test_pair_gradient_matches_finite_differences():
    dhat, kappa = 0.05, 1e3
    X, tets, body = _two_tets(0.01)
    X = X + 1e-3 * rng.normal(size=X.shape)
    faces = contact.boundary_faces(tets)
    edges = contact.face_edges(faces)
    pt, ee = contact.contact_pairs(X, faces, edges, body, dhat)
    assert len(pt) + len(ee) > 0
    g = contact.pair_gradient(X, faces, edges, pt, ee, kappa, dhat)
    e = 1e-7
    for v in range(len(X)):
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, c] += e
            Xm[v, c] -= e
            fd = (contact.pair_energy(Xp, faces, edges, pt, ee, kappa, dhat)
                  - contact.pair_energy(Xm, faces, edges, pt, ee, kappa, dhat)) / (2 * e)
            assert fd == pytest.approx(g[v, c], rel=1e-5, abs=1e-6 * np.abs(g).max())
    # Newton's third law: the pair forces sum to zero
    assert np.allclose(g.sum(axis=0), 0, atol=1e-9 * np.abs(g).max())


def test_ccd_exact_time_of_impact():
    """A point falling at constant speed onto a resting triangle from height
    h0 by a displacement 2 h0: with s = 0.1 the admissible fraction is the
    time at which the height is 0.1 h0, exactly (the rate bound is exact for
    a pure translation)."""
    f = lambda P: contact.point_triangle_distance(*P)
    xs0 = np.array([[0.2, 0.2, 0.8], [0, 0, 0], [1, 0, 0], [0, 1, 0]])
    dxs = np.zeros_like(xs0)
    dxs[0, 2] = -1.6
    assert contact.ccd_pair(f, xs0, dxs, 1, s=0.1) == pytest.approx(0.45, abs=1e-9)
    # moving away or parallel: the whole step
    dxs[0, 2] = +1.0
    assert contact.ccd_pair(f, xs0, dxs, 1) == 1.0
    # two edges closing head on: distance 1 shrinking at rate 4 -> 0.1 at t = 0.225
    g = lambda P: contact.edge_edge_distance(*P)
    xs = np.array([[0, 0, 0], [1, 0, 0], [0.5, -1, 1], [0.5, 1, 1]], dtype=np.float64)
    dx = np.array([[0, 0, 2], [0, 0, 2], [0, 0, -2], [0, 0, -2]], dtype=np.float64)
    assert contact.ccd_pair(g, xs, dx, 2, s=0.1) == pytest.approx(0.225, abs=1e-9)


def test_ccd_step_keeps_every_pair_apart():
    """Random displacements of two nearby tets closing on each other: along
    the returned fraction of the step, no point-triangle or edge-edge pair of
    different bodies gets closer than s times its starting distance (checked
    on a fine sampling of the path).  The fraction is conservative: the rate
    bound over-estimates how fast rotating primitives close, so the cut may
    come before the first sampled violation, never after it."""
    s = 0.1
    for trial in range(4):
        X, tets, body = _two_tets(0.02)
        faces = contact.boundary_faces(tets)
        edges = contact.face_edges(faces)
        dx = np.zeros_like(X)
        dx[4:] = np.array([0.0, 0.0, -0.3]) + 0.05 * rng.normal(size=(4, 3))
        alpha = contact.ccd_step(X, dx, faces, edges, body, s=s)
        assert 0 < alpha < 1

        def min_ratio(t):
            r = np.inf
            Xt = X + t * dx
            for v in np.unique(faces):
                for f in faces:
                    if body[v] != body[f[0]]:
                        r = min(r, contact.point_triangle_distance(Xt[v], *Xt[f])
                                / contact.point_triangle_distance(X[v], *X[f]))
            for i in range(len(edges)):
                for j in range(i + 1, len(edges)):
                    if body[edges[i][0]] != body[edges[j][0]]:
                        r = min(r, contact.edge_edge_distance(*Xt[edges[i]], *Xt[edges[j]])
                                / contact.edge_edge_distance(*X[edges[i]], *X[edges[j]]))
            return r

        assert min(min_ratio(t) for t in np.linspace(0, alpha, 25)) >= s * (1 - 1e-9)
        ts = np.linspace(0, 1, 201)
        bad = [t for t in ts if min_ratio(t) < s]
        assert not bad or alpha <= bad[0]


def _configs():
    """Point-triangle and edge-edge pairs whose closest features are, in
    turn, the plane / the two lines, a line, and a point."""
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    yield "pt", np.vstack([[0.2, 0.3, 0.05], tri])                 # over the face
    yield "pt", np.vstack([[0.5, -0.2, 0.05], tri])                # beside edge 0-1
    yield "pt", np.vstack([[-0.2, -0.1, 0.05], tri])               # beyond vertex 0
    yield "ee", np.array([[0, 0, 0], [1, 0, 0], [0.4, -1, 0.05], [0.6, 1, 0.05]], dtype=np.float64)
    yield "ee", np.array([[0, 0, 0], [1, 0, 0], [1.2, -1, 0.05], [1.3, 1, 0.05]], dtype=np.float64)
    yield "ee", np.array([[0, 0, 0], [1, 0, 0], [1.2, 0.1, 0.05], [2.0, 0.5, 0.05]], dtype=np.float64)


@pytest.mark.parametrize("case", range(6))
def test_pair_distance_derivatives_match_finite_differences(case):
    kind, X = list(_configs())[case]
    X = X + 1e-4 * rng.normal(size=X.shape)
    dist = (lambda Y: contact.point_triangle_distance(*Y.reshape(4, 3))) if kind == "pt" else \
        (lambda Y: contact.edge_edge_distance(*Y.reshape(4, 3)))
    d, g, H = contact.pair_distance_derivatives(kind, X)
    x = X.ravel()
    assert d == pytest.approx(dist(x), rel=1e-13)
    e = 1e-6
    E = np.eye(12)
    fd = np.array([(dist(x + e * E[k]) - dist(x - e * E[k])) / (2 * e) for k in range(12)])
    assert np.allclose(fd, g, rtol=0, atol=1e-8)
    gfun = lambda Y: contact.pair_distance_derivatives(kind, Y.reshape(4, 3))[1]
    fdH = np.array([(gfun(x + e * E[k]) - gfun(x - e * E[k])) / (2 * e) for k in range(12)])
    assert np.allclose(fdH, H, rtol=0, atol=1e-5 * max(np.abs(H).max(), 1.0))
    assert np.allclose(H, H.T, atol=1e-14 * max(np.abs(H).max(), 1.0))
    # a rigid translation changes no distance
    for c in range(3):
        t = np.tile(np.eye(3)[c], 4)
        assert abs(g @ t) <= 1e-12 and np.abs(H @ t).max() <= 1e-9 * max(np.abs(H).max(), 1.0)


def test_pair_barrier_hessian_is_the_gradients_derivative_then_projected():
    kind, X = list(_configs())[0]
    dhat, kappa = 0.1, 1e3
    faces = np.array([[1, 2, 3]])
    edges = np.zeros((0, 2), dtype=np.int64)
    H = contact.pair_barrier_hessian(kind, X, kappa, dhat, project=False)
    e = 1e-7
    x = X.ravel()
    gb = lambda Y: contact.pair_gradient(Y.reshape(4, 3), faces, edges, [(0, 0)], [], kappa, dhat).ravel()
    fdH = np.array([(gb(x + e * np.eye(12)[k]) - gb(x - e * np.eye(12)[k])) / (2 * e) for k in range(12)])
    assert np.allclose(fdH, H, rtol=1e-5, atol=1e-6 * np.abs(H).max())
    Hp = contact.pair_barrier_hessian(kind, X, kappa, dhat)
    w = np.linalg.eigvalsh(Hp)
    assert w.min() >= -1e-9 * w.max() and np.allclose(Hp, Hp.T)
    # the projection keeps the non-negative part of the spectrum
    w0 = np.linalg.eigvalsh(H)
    assert np.allclose(np.sort(w), np.sort(np.maximum(w0, 0)), atol=1e-9 * np.abs(w0).max())


def test_problem_with_mesh_contact_gradient_and_collision_step():
    """Eq. IP with the mesh-mesh barrier: the gradient is the derivative of
    E near contact, and a step of a block driven into another ends at a
    minimiser with the blocks apart, where the same step without the
    barrier passes one into the other."""
    import synth
    from oracle import ip, newton
    s, body = synth.two_block_scene(gap=0.004, speed=0.6)
    p = ip.Problem(s, body=body)
    n0 = int((body == 0).sum())
    # near contact: the upper block lowered to 0.5 mm above the lower one
    x = s.x0.copy()
    x[n0:, 2] -= 0.0035
    x += 1e-5 * rng.normal(size=x.shape)
    pt, ee = p.pairs(x)
    assert pt or ee
    g = p.gradient(x)
    e = 1e-8
    near = np.unique([v for v, _ in pt] + [int(w) for i, j in ee for w in (*p.edges[i], *p.edges[j])])
    for v in list(near[:6]) + [0, len(x) - 1]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += e
            xm[v, c] -= e
            fd = (p.energy(xp) - p.energy(xm)) / (2 * e)
            assert fd == pytest.approx(g[v, c], rel=1e-4, abs=1e-6 * np.abs(g).max())
    H = p.hessian(x).toarray()
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0
    # the collision step
    x1, info = newton.timestep(p)
    assert p.feasible(x1)
    assert np.abs(p.gradient(x1)).max() <= 1e-6 * max(np.abs(p.gradient(s.x0)).max(), 1e-300) + 1e-9
    assert _vertices_inside_other_body(x1, s.tets, body) == 0
    x_free, _ = newton.timestep(ip.Problem(s))
    assert _vertices_inside_other_body(x_free, s.tets, body) > 0



def test_final_newton_direction_is_ccd_filtered_between_bodies():
    """Sec. 3.9: every update of the iterate passes the CCD filter, the
    final small Newton direction too.  A move that carries a vertex of one
    tet through the other's top face ends with no touching pair, so the
    feasibility test alone would accept it; the mesh-mesh filter rejects
    it and lets the opposite move through.  Without bodies nothing is cut."""
    from types import SimpleNamespace
    from oracle import newton
    gap = 1e-4
    X, tets, body = _two_tets(gap)
    faces = contact.boundary_faces(tets)
    edges = contact.face_edges(faces)
    prob = SimpleNamespace(body=body, faces=faces, edges=edges)
    d = np.zeros_like(X)
    d[4:, 2] = -2 * gap
    pt, ee = contact.contact_pairs(X + d, faces, edges, body, 1e-300)
    assert not pt and not ee
    assert _vertices_inside_other_body(X + d, tets, body) == 1
    assert not newton._uncut_between_bodies(prob, X, d)
    assert newton._uncut_between_bodies(prob, X, -d)
    assert newton._uncut_between_bodies(SimpleNamespace(body=None), X, d)

def _vertices_inside_other_body(x, tets, body):
    """How many vertices lie strictly inside a tet of another body."""
    count = 0
    for v in range(len(x)):
        for t in tets:
            if body[t[0]] == body[v]:
                continue
            T = np.stack([x[t[1]] - x[t[0]], x[t[2]] - x[t[0]], x[t[3]] - x[t[0]]], axis=1)
            lam = np.linalg.solve(T, x[v] - x[t[0]])
            if lam.min() > 0 and lam.sum() < 1:
                count += 1
                break
    return count
