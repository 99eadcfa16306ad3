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
