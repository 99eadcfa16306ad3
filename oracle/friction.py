"""Lagged, mollified friction for point-plane contact (oracle).

The paper's friction term D in Eq. IP is the IPC frictional pseudo-potential
(Sec. 3.1, cited, not written out).  The reading used here, for the ground
plane with unit normal n and a vertex k in contact at the lagged state x^lag
(distance d_k < dhat):

    lambda_k = -kappa b'(d_k(x^lag)) >= 0   (the lagged normal force magnitude,
                                             b the point-plane barrier)
    T        = an orthonormal basis (3 x 2) of the plane's tangent space
    u_k(x)   = T^T (x_k - x_k^t)            (tangential displacement over the step)
    D(x)     = sum_k mu lambda_k f0(|u_k|)

with the C1 mollifier of width eps = eps_v h (eps_v a velocity):

    f1(y) = 2 y / eps - y^2 / eps^2  for y < eps,   1 for y >= eps,
    f0(y) = -y^3 / (3 eps^2) + y^2 / eps + eps / 3   for y < eps,   y for y >= eps,

so f0' = f1, f0 and f1 are continuous at eps, and a sliding vertex
(|u| >= eps) feels the Coulomb force of magnitude mu lambda_k.  D enters E
with the same alpha h^2 factor as the elastic energy.  Per vertex the
Hessian is mu lambda T (f1'(y) u^ u^T + f1(y)/y (I - u^ u^T)) T^T (u^ = u / y),
positive semi-definite because f1' >= 0 and f1 >= 0 on y >= 0; at y = 0 it is
mu lambda (2 / eps) T T^T.  The lag state is x^t (one normal-force and
tangent update per timestep).
"""
from __future__ import annotations

import numpy as np

from . import barrier


def f0(y, eps):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, -y ** 3 / (3.0 * eps ** 2) + y ** 2 / eps + eps / 3.0, y)


def f1(y, eps):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, 2.0 * y / eps - y ** 2 / eps ** 2, 1.0)


def df1(y, eps):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, 2.0 / eps - 2.0 * y / eps ** 2, 0.0)


def tangent_basis(n):
    """Orthonormal 3 x 2 basis of the plane with unit normal n."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    t1 = a - n * (a @ n)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    return np.stack([t1, t2], axis=1)


class GroundFriction:
    """D(x) for one timestep: normal forces and tangent basis lagged at x_lag."""

    def __init__(self, mu, eps_v, h, kappa, dhat, plane_n, plane_o, x_t, x_lag=None):
        self.mu = float(mu)
        self.eps = float(eps_v) * float(h)
        self.x_t = np.asarray(x_t, dtype=np.float64)
        x_lag = self.x_t if x_lag is None else np.asarray(x_lag, dtype=np.float64)
        n = np.asarray(plane_n, dtype=np.float64)
        d = x_lag @ n - float(plane_o)
        self.lam = -float(kappa) * barrier.db(d, dhat)          # >= 0, zero outside contact
        self.T = tangent_basis(n)

    def _u(self, x):
        return (np.asarray(x, dtype=np.float64) - self.x_t) @ self.T   # [n, 2]

    def energy(self, x):
        y = np.linalg.norm(self._u(x), axis=1)
        return float(np.sum(self.mu * self.lam * f0(y, self.eps)))

    def gradient(self, x):
        """dD/dx [n, 3]."""
        u = self._u(x)
        y = np.linalg.norm(u, axis=1)
        # f1(y) / y, with its limit 2 / eps at y = 0
        ratio = np.where(y > 0, f1(y, self.eps) / np.where(y > 0, y, 1.0), 2.0 / self.eps)
        return (self.mu * self.lam * ratio)[:, None] * (u @ self.T.T)

    def hessian_blocks(self, x):
        """d2D/dx_k^2 per vertex [n, 3, 3] (D couples no two vertices)."""
        u = self._u(x)
        y = np.linalg.norm(u, axis=1)
        safe = np.where(y > 0, y, 1.0)
        uh = u / safe[:, None]
        ratio = np.where(y > 0, f1(y, self.eps) / safe, 2.0 / self.eps)
        slope = np.where(y > 0, df1(y, self.eps), 2.0 / self.eps)
        I2 = np.eye(2)[None]
        P = uh[:, :, None] * uh[:, None, :]
        K2 = slope[:, None, None] * P + ratio[:, None, None] * (I2 - P)   # at y = 0 both give (2/eps) I
        K3 = self.T[None] @ K2 @ self.T.T[None]
        return (self.mu * self.lam)[:, None, None] * K3


class PairFriction:
    """Lagged, mollified friction between surface primitives of different
    bodies (Eq. IP term D for mesh-mesh contact), the same construction as
    the ground term above with the plane replaced by each pair's closest
    points.  Reading, at the lag state x^lag = x^t, for every point-triangle
    and edge-edge pair of different bodies closer than dhat (contact.py):

        y_k - z_k = sum_j w_kj x_j   the closest-point difference, w_k the
                                     closest points' weights on the pair's
                                     four vertices: (1, -beta_a, -beta_b,
                                     -beta_c) for point-triangle, (1 - s, s,
                                     -(1 - t), -t) for edge-edge; sum_j w_kj = 0
        n_k      = (y_k - z_k) / d_k, d_k = |y_k - z_k|
        lambda_k = -kappa b'(d_k) >= 0
        u_k(x)   = (I - n_k n_k^T) sum_j w_kj (x_j - x_j^t)
        D(x)     = sum_k mu lambda_k f0(|u_k|)

    w, n and lambda stay fixed over the timestep, so u_k is the relative
    tangential displacement of the two closest points over the step.  Written
    with the projector I - n n^T, no tangent basis is needed: |u| equals
    |T^T r| for any orthonormal basis T of the plane normal to n.  The pair's
    12 x 12 Hessian is w_k w_k^T (x) mu lambda_k K_k with the 3 x 3
    K = (f1(y)/y) (I - n n^T) + (f1'(y) - f1(y)/y) u^ u^T (u^ = u / y), which is
    positive semi-definite (f1 >= 0, f1' >= 0; at y = 0, K = (2 / eps)
    (I - n n^T)), and so is w w^T."""

    def __init__(self, mu, eps_v, h, kappa, dhat, faces, edges, body, x_t, x_lag=None):
        from . import contact
        self.mu = float(mu)
        self.eps = float(eps_v) * float(h)
        self.x_t = np.asarray(x_t, dtype=np.float64)
        x_lag = self.x_t if x_lag is None else np.asarray(x_lag, dtype=np.float64)
        pt, ee = contact.contact_pairs(x_lag, faces, edges, body, dhat)
        vids, w, n, d = [], [], [], []
        for v, k in pt:
            a, b, c = x_lag[faces[k]]
            q = contact.closest_point_triangle(x_lag[v], a, b, c)
            beta = contact._triangle_weights(q, a, b, c)
            vids.append([v, *faces[k]])
            w.append([1.0, -beta[0], -beta[1], -beta[2]])
            n.append(x_lag[v] - q)
        for i, j in ee:
            p0, p1 = x_lag[edges[i]]
            q0, q1 = x_lag[edges[j]]
            y, z = contact.closest_points_segments(p0, p1, q0, q1)
            s = contact._segment_weight(y, p0, p1)
            t = contact._segment_weight(z, q0, q1)
            vids.append([*edges[i], *edges[j]])
            w.append([1.0 - s, s, -(1.0 - t), -t])
            n.append(y - z)
        self.vids = np.asarray(vids, dtype=np.int64).reshape(-1, 4)
        self.w = np.asarray(w, dtype=np.float64).reshape(-1, 4)
        n = np.asarray(n, dtype=np.float64).reshape(-1, 3)
        d = np.linalg.norm(n, axis=1)
        self.n = n / np.where(d > 0, d, 1.0)[:, None]
        self.lam = -float(kappa) * barrier.db(d, dhat)
        self.n_pt = len(pt)

    def _u(self, x):
        x = np.asarray(x, dtype=np.float64)
        r = np.einsum("kj,kjc->kc", self.w, x[self.vids] - self.x_t[self.vids])
        return r - self.n * np.sum(r * self.n, axis=1, keepdims=True)

    def energy(self, x):
        y = np.linalg.norm(self._u(x), axis=1)
        return float(np.sum(self.mu * self.lam * f0(y, self.eps)))

    def gradient(self, x):
        """dD/dx [n, 3]: vertex j of pair k gains mu lambda_k (f1(y)/y) w_kj u_k."""
        u = self._u(x)
        y = np.linalg.norm(u, axis=1)
        ratio = np.where(y > 0, f1(y, self.eps) / np.where(y > 0, y, 1.0), 2.0 / self.eps)
        gk = (self.mu * self.lam * ratio)[:, None, None] * self.w[:, :, None] * u[:, None, :]   # [P, 4, 3]
        g = np.zeros_like(self.x_t)
        np.add.at(g, self.vids.ravel(), gk.reshape(-1, 3))
        return g

    def hessian_pairs(self, x):
        """d2D/dx2 of each pair over its four vertices [P, 12, 12]."""
        u = self._u(x)
        y = np.linalg.norm(u, axis=1)
        safe = np.where(y > 0, y, 1.0)
        uh = u / safe[:, None]
        ratio = np.where(y > 0, f1(y, self.eps) / safe, 2.0 / self.eps)
        slope = np.where(y > 0, df1(y, self.eps), 2.0 / self.eps)
        Pn = np.eye(3)[None] - self.n[:, :, None] * self.n[:, None, :]
        K = ratio[:, None, None] * Pn + (slope - ratio)[:, None, None] * (uh[:, :, None] * uh[:, None, :])
        ww = self.w[:, :, None] * self.w[:, None, :]                                            # [P, 4, 4]
        H = (self.mu * self.lam)[:, None, None, None, None] * ww[:, :, None, :, None] * K[:, None, :, None, :]
        return H.reshape(-1, 12, 12)
