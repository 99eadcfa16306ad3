"""Mesh-mesh contact primitives (oracle): distances, barrier, CCD.

The paper models contact with IPC barriers (Sec. 3.1, Eq. IP term B, and
Sec. 3.9's filtered line search with CCD), cited, not written out.  This
module is the oracle for the mesh-mesh part of that term: point-triangle
and edge-edge pairs between surface primitives of different objects.
Readings:

* the barrier acts on the unsquared distance d with the same
  b(d) = -(d - dhat)^2 ln(d / dhat) as the point-plane term (barrier.py);
* a pair's distance is the Euclidean distance between the closest points of
  the two primitives (closed segments, closed triangles): the plane
  projection or the nearest edge for a triangle, and the best of the
  interior stationary point and the four boundary optima for two segments;
* no mollifier for nearly parallel edge pairs (the workloads here have no
  such pairs at contact distance);
* CCD is conservative advancement with the additive-CCD rate bound:
  primitives move linearly over the step; L, the sum of the two primitives'
  largest vertex displacements relative to a common translation, bounds the
  rate of change of their distance, and the fraction advances by
  (d(t) - s d0) / L until it converges or reaches 1 (s = 0.1 by default),
  so the pair never comes closer than s times its starting distance.
"""
from __future__ import annotations

import numpy as np

from . import barrier


# ---- closest points ---------------------------------------------------------------------------
def _closest_on_segment(p, a, b):
    """Closest point to p on the closed segment ab: the clamped projection."""
    d = b - a
    L = d @ d
    if L <= 0:
        return a
    return a + np.clip((p - a) @ d / L, 0.0, 1.0) * d


def closest_point_triangle(p, a, b, c):
    """Closest point to p on the closed triangle abc.  The projection of p on
    the triangle's plane is the answer when its barycentric coordinates are
    all non-negative; otherwise the closest point lies on the boundary, and
    it is the nearest of the three edges' clamped projections."""
    p, a, b, c = (np.asarray(v, dtype=np.float64) for v in (p, a, b, c))
    n = np.cross(b - a, c - a)
    nn = n @ n
    if nn > 0:
        q = p - ((p - a) @ n / nn) * n
        # barycentric coordinates from sub-triangle areas (signed by n)
        wa = np.cross(b - q, c - q) @ n / nn
        wb = np.cross(c - q, a - q) @ n / nn
        wc = 1.0 - wa - wb
        if wa >= 0 and wb >= 0 and wc >= 0:
            return q
    cands = [_closest_on_segment(p, a, b), _closest_on_segment(p, b, c), _closest_on_segment(p, c, a)]
    return min(cands, key=lambda y: (p - y) @ (p - y))


def closest_points_segments(p0, p1, q0, q1):
    """Closest points (on p0p1, on q0q1) of two closed segments: the minimum
    of |p0 + s d1 - q0 - t d2|^2 over the unit square, taken among the
    interior stationary point (when the 2 x 2 normal equations are regular
    and it lies inside) and the optima on the square's four sides."""
    p0, p1, q0, q1 = (np.asarray(v, dtype=np.float64) for v in (p0, p1, q0, q1))
    d1, d2 = p1 - p0, q1 - q0
    cands = []
    A = np.array([[d1 @ d1, -(d1 @ d2)], [-(d1 @ d2), d2 @ d2]])
    rhs = np.array([(q0 - p0) @ d1, -((q0 - p0) @ d2)])
    if abs(np.linalg.det(A)) > 1e-14 * max(abs(A).max() ** 2, 1e-300):
        st = np.linalg.solve(A, rhs)
        if 0 <= st[0] <= 1 and 0 <= st[1] <= 1:
            cands.append((p0 + st[0] * d1, q0 + st[1] * d2))
    for s_fix in (0.0, 1.0):                       # s on a side: best t by clamped projection
        y = p0 + s_fix * d1
        cands.append((y, _closest_on_segment(y, q0, q1)))
    for t_fix in (0.0, 1.0):                       # t on a side: best s
        z = q0 + t_fix * d2
        cands.append((_closest_on_segment(z, p0, p1), z))
    return min(cands, key=lambda yz: (yz[0] - yz[1]) @ (yz[0] - yz[1]))


def point_triangle_distance(p, a, b, c):
    return float(np.linalg.norm(np.asarray(p, dtype=np.float64) - closest_point_triangle(p, a, b, c)))


def edge_edge_distance(p0, p1, q0, q1):
    x, y = closest_points_segments(p0, p1, q0, q1)
    return float(np.linalg.norm(x - y))


# ---- surface and pairs ----------------------------------------------------------------------
def boundary_faces(tets):
    """Faces of a tet mesh that belong to one tet only, oriented outward-agnostic
    (vertex order as in the tet), [f, 3]."""
    tets = np.asarray(tets, dtype=np.int64)
    faces = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]])
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return faces[cnt[inv.ravel()] == 1]


def face_edges(faces):
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    return np.unique(np.sort(e, axis=1), axis=0)


def contact_pairs(x, faces, edges, body, dhat):
    """All point-triangle (vertex, face) and edge-edge (edge, edge) pairs of
    different bodies closer than dhat, by brute force.  ``body`` [n] labels
    the body of each vertex."""
    x = np.asarray(x, dtype=np.float64)
    verts = np.unique(faces)
    pt, ee = [], []
    for v in verts:
        for k, f in enumerate(faces):
            if body[v] == body[f[0]]:
                continue
            if point_triangle_distance(x[v], *x[f]) < dhat:
                pt.append((v, k))
    for i in range(len(edges)):
        for j in range(i + 1, len(edges)):
            ei, ej = edges[i], edges[j]
            if body[ei[0]] == body[ej[0]]:
                continue
            if edge_edge_distance(*x[ei], *x[ej]) < dhat:
                ee.append((i, j))
    return pt, ee


# ---- barrier energy and gradient ----------------------------------------------------------------
def pair_energy(x, faces, edges, pt, ee, kappa, dhat):
    """kappa sum over pairs of b(d); +inf if any pair touches."""
    x = np.asarray(x, dtype=np.float64)
    d = [point_triangle_distance(x[v], *x[faces[k]]) for v, k in pt]
    d += [edge_edge_distance(*x[edges[i]], *x[edges[j]]) for i, j in ee]
    return float(kappa * np.sum(barrier.b(np.asarray(d), dhat))) if d else 0.0


def pair_gradient(x, faces, edges, pt, ee, kappa, dhat):
    """dB/dx [n, 3].  With closest points y on one primitive and z on the
    other, d = |y - z| and the gradient of d with respect to each vertex is
    its barycentric weight in y (or z) times +-(y - z)/d; the weights are
    those of the closest point, which is stationary in them (envelope)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros_like(x)
    for v, k in pt:
        a, b, c = x[faces[k]]
        q = closest_point_triangle(x[v], a, b, c)
        d = np.linalg.norm(x[v] - q)
        w = _triangle_weights(q, a, b, c)
        gd = (x[v] - q) / d
        s = kappa * barrier.db(np.array([d]), dhat)[0]
        g[v] += s * gd
        for wi, vi in zip(w, faces[k]):
            g[vi] -= s * wi * gd
    for i, j in ee:
        p0, p1 = x[edges[i]]
        q0, q1 = x[edges[j]]
        y, z = closest_points_segments(p0, p1, q0, q1)
        d = np.linalg.norm(y - z)
        gd = (y - z) / d
        s = kappa * barrier.db(np.array([d]), dhat)[0]
        sp = _segment_weight(y, p0, p1)
        sq = _segment_weight(z, q0, q1)
        g[edges[i][0]] += s * (1 - sp) * gd
        g[edges[i][1]] += s * sp * gd
        g[edges[j][0]] -= s * (1 - sq) * gd
        g[edges[j][1]] -= s * sq * gd
    return g


def _triangle_weights(q, a, b, c):
    """Barycentric weights of a point q of the triangle abc."""
    T = np.stack([b - a, c - a], axis=1)
    uv, *_ = np.linalg.lstsq(T, q - a, rcond=None)
    return np.array([1.0 - uv.sum(), uv[0], uv[1]])


def _segment_weight(y, p0, p1):
    d = p1 - p0
    L = d @ d
    return 0.0 if L <= 0 else float(np.clip((y - p0) @ d / L, 0.0, 1.0))


# ---- continuous collision detection -------------------------------------------------------------
def ccd_pair(dist, xs0, dxs, split, s=0.1, max_iter=100000, rtol=1e-10):
    """Conservative advancement for one primitive pair whose vertices move
    linearly: xs0 [k, 3] start positions, dxs [k, 3] displacements, the
    first ``split`` rows the first primitive's vertices; dist(positions) ->
    the pair's distance.  The distance changes at rate at most L, the sum
    over the two primitives of their largest vertex displacement relative to
    a common translation (the additive CCD bound).  From distance d at t,
    the fraction t + (d - s d0) / L therefore keeps the distance >= s d0;
    the steps shrink as d approaches s d0.  Returns the fraction reached
    (1 if the whole step keeps the distance >= s d0)."""
    xs0 = np.asarray(xs0, dtype=np.float64)
    dxs = np.asarray(dxs, dtype=np.float64)
    rel = dxs - dxs.mean(axis=0)
    L = np.max(np.linalg.norm(rel[:split], axis=1)) + np.max(np.linalg.norm(rel[split:], axis=1))
    d0 = dist(xs0)
    if L <= 0:
        return 1.0
    floor = s * d0
    t, d = 0.0, d0
    for _ in range(max_iter):
        step = (d - floor) / L
        if step <= rtol:
            return t
        if t + step >= 1.0:
            return 1.0 if dist(xs0 + dxs) >= floor * (1 - 1e-12) else t
        d_next = dist(xs0 + (t + step) * dxs)
        if d_next < floor * (1 - 1e-12):     # only rounding can cause this
            return t
        t, d = t + step, d_next
    return t


def ccd_step(x, dx, faces, edges, body, s=0.1):
    """Largest fraction alpha in [0, 1] of the step dx for which no
    point-triangle or edge-edge pair of different bodies comes closer than s
    times its starting distance (brute force over all such pairs)."""
    x = np.asarray(x, dtype=np.float64)
    dx = np.asarray(dx, dtype=np.float64)
    alpha = 1.0
    verts = np.unique(faces)
    for v in verts:
        for f in faces:
            if body[v] == body[f[0]]:
                continue
            idx = np.array([v, *f])
            alpha = min(alpha, ccd_pair(lambda P: point_triangle_distance(*P), x[idx], dx[idx], 1, s))
    for i in range(len(edges)):
        for j in range(i + 1, len(edges)):
            if body[edges[i][0]] == body[edges[j][0]]:
                continue
            idx = np.array([*edges[i], *edges[j]])
            alpha = min(alpha, ccd_pair(lambda P: edge_edge_distance(*P), x[idx], dx[idx], 2, s))
    return alpha


# ---- exact second derivatives: hyper-dual numbers ------------------------------------------------
class _HD:
    """Hyper-dual number r + a e1 + b e2 + c e1 e2 (e1^2 = e2^2 = 0): evaluating
    f at x + e1 u + e2 v gives f(x), the directional derivatives along u and
    v, and u^T (d2 f) v exactly, with no truncation error."""

    __slots__ = ("r", "a", "b", "c")

    def __init__(self, r, a=0.0, b=0.0, c=0.0):
        self.r, self.a, self.b, self.c = r, a, b, c

    def __add__(self, o):
        if not isinstance(o, _HD):
            return _HD(self.r + o, self.a, self.b, self.c)
        return _HD(self.r + o.r, self.a + o.a, self.b + o.b, self.c + o.c)

    __radd__ = __add__

    def __neg__(self):
        return _HD(-self.r, -self.a, -self.b, -self.c)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not isinstance(o, _HD):
            return _HD(self.r * o, self.a * o, self.b * o, self.c * o)
        return _HD(self.r * o.r, self.r * o.a + self.a * o.r, self.r * o.b + self.b * o.r,
                   self.r * o.c + self.a * o.b + self.b * o.a + self.c * o.r)

    __rmul__ = __mul__

    def inv(self):
        r = 1.0 / self.r
        return _HD(r, -self.a * r * r, -self.b * r * r, -self.c * r * r + 2.0 * self.a * self.b * r * r * r)

    def __truediv__(self, o):
        return self * (o.inv() if isinstance(o, _HD) else 1.0 / o)

    def sqrt(self):
        s = np.sqrt(self.r)
        return _HD(s, self.a / (2 * s), self.b / (2 * s), self.c / (2 * s) - self.a * self.b / (4 * s * s * s))


def _dot(u, v):
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]


def _cross(u, v):
    return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]


def _sub(u, v):
    return [u[k] - v[k] for k in range(3)]


def _norm(u):
    return _dot(u, u).sqrt()


def _d_pp(P):            # point-point
    return _norm(_sub(P[0], P[1]))


def _d_pe(P):            # point P0 to the line through P1 P2
    e = _sub(P[2], P[1])
    return _norm(_cross(_sub(P[0], P[1]), e)) / _norm(e)


def _d_pt(P, sgn):       # point P0 to the plane of P1 P2 P3 (sgn: side of P0)
    n = _cross(_sub(P[2], P[1]), _sub(P[3], P[1]))
    return _dot(_sub(P[0], P[1]), n) * sgn / _norm(n)


def _d_ee(P, sgn):       # line P0 P1 to line P2 P3 (sgn: sign of the triple product)
    n = _cross(_sub(P[1], P[0]), _sub(P[3], P[2]))
    return _dot(_sub(P[2], P[0]), n) * sgn / _norm(n)


def _derivatives(fn, X):
    """Value, gradient and Hessian of fn over the stacked coordinates of the
    vertices X [k, 3], evaluated once on (m x m) arrays of hyper-dual parts."""
    X = np.asarray(X, dtype=np.float64)
    m = X.size
    I = np.eye(m)
    ones = np.ones(m)
    flat = X.ravel()
    P = [[_HD(np.full((m, m), flat[3 * i + c]), np.outer(I[:, 3 * i + c], ones), np.outer(ones, I[:, 3 * i + c]),
              np.zeros((m, m))) for c in range(3)] for i in range(len(X))]
    f = fn(P)
    return float(f.r[0, 0]), f.a[:, 0].copy(), 0.5 * (f.c + f.c.T)


def _pt_type(p, a, b, c):
    """The closest feature of triangle abc to p: ('pt',), ('pe', i, j) or ('pp', i)
    with local indices 0..2 of the triangle's vertices."""
    q = closest_point_triangle(p, a, b, c)
    w = _triangle_weights(q, a, b, c)
    zero = np.abs(w) <= 1e-12
    if not zero.any():
        return ("pt",)
    if zero.sum() == 1:
        i, j = [k for k in range(3) if not zero[k]]
        return ("pe", i, j)
    return ("pp", int(np.argmax(w)))


def _ee_type(p0, p1, q0, q1):
    """('ee',) or a reduced pair: ('pe', point, seg_a, seg_b) / ('pp', i, j)
    with local indices 0..3 (p0, p1, q0, q1)."""
    y, z = closest_points_segments(p0, p1, q0, q1)
    s = _segment_weight(y, p0, p1)
    t = _segment_weight(z, q0, q1)
    s_end = s <= 1e-12 or s >= 1 - 1e-12
    t_end = t <= 1e-12 or t >= 1 - 1e-12
    if not s_end and not t_end:
        return ("ee",)
    if s_end and t_end:
        return ("pp", 0 if s < 0.5 else 1, 2 if t < 0.5 else 3)
    if s_end:
        return ("pe", 0 if s < 0.5 else 1, 2, 3)
    return ("pe", 2 if t < 0.5 else 3, 0, 1)


def pair_distance_derivatives(kind, X):
    """Distance of a point-triangle (kind 'pt', X = [p, a, b, c]) or
    edge-edge (kind 'ee', X = [p0, p1, q0, q1]) pair with its gradient and
    Hessian over the 12 stacked coordinates, from the formula of the closest
    feature (plane, line or point) evaluated in hyper-dual numbers."""
    X = np.asarray(X, dtype=np.float64)
    if kind == "pt":
        t = _pt_type(*X)
        if t[0] == "pt":
            n = np.cross(X[2] - X[1], X[3] - X[1])
            sgn = 1.0 if (X[0] - X[1]) @ n >= 0 else -1.0
            return _derivatives(lambda P: _d_pt(P, sgn), X)
        idx = [0, 1 + t[1], 1 + t[2]] if t[0] == "pe" else [0, 1 + t[1]]
    else:
        t = _ee_type(*X)
        if t[0] == "ee":
            n = np.cross(X[1] - X[0], X[3] - X[2])
            sgn = 1.0 if (X[2] - X[0]) @ n >= 0 else -1.0
            return _derivatives(lambda P: _d_ee(P, sgn), X)
        idx = list(t[1:])
    sub = X[idx]
    val, g_sub, H_sub = _derivatives(_d_pe if len(idx) == 3 else _d_pp, sub)
    g = np.zeros(12)
    H = np.zeros((12, 12))
    cols = np.concatenate([np.arange(3 * k, 3 * k + 3) for k in idx])
    g[cols] = g_sub
    H[np.ix_(cols, cols)] = H_sub
    return val, g, H


def pair_barrier_hessian(kind, X, kappa, dhat, project=True):
    """kappa (b''(d) grad d grad d^T + b'(d) Hess d) over the pair's 12
    coordinates, projected to the positive semi-definite cone per pair
    (eigenvalues clamped at zero) unless project is False."""
    d, g, Hd = pair_distance_derivatives(kind, X)
    da = np.array([d])
    H = kappa * (barrier.d2b(da, dhat)[0] * np.outer(g, g) + barrier.db(da, dhat)[0] * Hd)
    if project:
        w, V = np.linalg.eigh(0.5 * (H + H.T))
        H = (V * np.maximum(w, 0.0)) @ V.T
    return H
