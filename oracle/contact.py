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
