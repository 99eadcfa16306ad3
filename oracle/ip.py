"""Incremental potential for one timestep (oracle).

Eq. IP (Sec. 3.1) with implicit Euler: alpha = 1, predictor
x_tilde = x^t + h v^t, velocity update v^{t+1} = (x^{t+1} - x^t) / h; or
with BDF2: alpha = 4/9, x_tilde = (4 x^t - x^{t-1}) / 3 + (2h/9)(4 v^t -
v^{t-1}), v^{t+1} = (4 v^t - v^{t-1}) / 3 + (2h/3) a^{t+1}.  The printed
acceleration a^{t+1} = (4h^2/9)(x^{t+1} - x_tilde) is dimensionally garbled;
the reading a^{t+1} = (9 / (4 h^2)) (x^{t+1} - x_tilde) is the one that makes
x_tilde + (4h^2/9) a^{t+1} = x^{t+1} (the BDF2 position update), and with it
v^{t+1} = (3 x^{t+1} - 4 x^t + x^{t-1}) / (2h), the BDF2 velocity.
Readings used where the paper is silent:

* mass: lumped, m_v = sum over tets e containing v of rho_e vol_e / 4;
* gravity g enters through the predictor, x_tilde += alpha h^2 g
  (equivalent to the potential -M g . x in the alpha h^2-scaled bracket);
* friction D = 0 unless ``mu`` > 0 is given (no workload uses friction);
  then D is the lagged, mollified point-plane friction of ``friction.py``
  and, with bodies, its mesh-mesh form between their surface primitives
  (``friction.PairFriction``);
* Dirichlet vertices are held at x^t: they are not unknowns, their inertia
  term is dropped, their gradient entries are zero and their Hessian rows
  and columns are the identity.

    E(x) = 1/2 sum_{v free} m_v |x_v - x_tilde_v|^2
           + alpha h^2 ( sum_e vol_e psi(F_e(x)) + kappa sum_v b(n . x_v - o) ).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import barrier, contact, elastic, friction


class Problem:
    """One timestep's incremental potential built from a synthetic scene."""

    def __init__(self, scene, x_t=None, v_t=None, dt=None, project=True, integrator="ie", x_prev=None,
                 v_prev=None, mu=0.0, eps_v=1e-3, body=None, threads=1):
        # threads > 1: the per-element terms are evaluated on contiguous
        # chunks of the tets by a thread pool and concatenated in tet order;
        # every element's arithmetic is the same as in one call
        self.threads = max(1, int(threads))
        self.X = np.asarray(scene.X, dtype=np.float64)
        self.tets = np.asarray(scene.tets, dtype=np.int64)
        self.n = self.X.shape[0]
        self.vol, self.Dm_inv = elastic.rest_shape(self.X, self.tets)
        self.mu, self.lam = elastic.lame(scene.E, scene.nu)
        rho = np.asarray(scene.rho, dtype=np.float64)
        self.mass = np.zeros(self.n)
        np.add.at(self.mass, self.tets.ravel(), np.repeat(rho * self.vol / 4.0, 4))
        self.pinned = np.asarray(scene.dirichlet).astype(bool)
        self.free = ~self.pinned
        self.h = float(scene.dt if dt is None else dt)
        self.gravity = np.asarray(scene.gravity, dtype=np.float64)
        self.contact = bool(scene.contact)
        self.plane_n = np.asarray(scene.plane_n, dtype=np.float64)
        self.plane_o = float(scene.plane_o)
        self.dhat = float(scene.dhat)
        self.kappa = float(scene.kappa)
        self.project = project
        self.x_t = np.array(scene.x0 if x_t is None else x_t, dtype=np.float64)
        self.v_t = np.array(scene.v0 if v_t is None else v_t, dtype=np.float64)
        self.integrator = integrator
        if integrator == "ie":
            self.alpha = 1.0
            self.x_tilde = self.x_t + self.h * self.v_t + self.h ** 2 * self.gravity[None, :]
        elif integrator == "bdf2":
            if x_prev is None or v_prev is None:
                raise ValueError("BDF2 needs x^{t-1} and v^{t-1}")
            self.alpha = 4.0 / 9.0
            self.x_prev = np.array(x_prev, dtype=np.float64)
            self.v_prev = np.array(v_prev, dtype=np.float64)
            self.x_tilde = ((4.0 * self.x_t - self.x_prev) / 3.0 + (2.0 * self.h / 9.0) * (4.0 * self.v_t - self.v_prev)
                            + self.alpha * self.h ** 2 * self.gravity[None, :])
        else:
            raise ValueError(f"unknown integrator {integrator!r}")
        self.ah2 = self.alpha * self.h ** 2   # the factor on the potentials
        self.x_tilde[self.pinned] = self.x_t[self.pinned]
        # mesh-mesh contact between the bodies ``body`` labels (contact.py)
        self.body = None if body is None else np.asarray(body, dtype=np.int64)
        if self.body is not None:
            self.faces = contact.boundary_faces(self.tets)
            self.edges = contact.face_edges(self.faces)
        self.friction = None
        if mu > 0 and self.contact:
            self.friction = friction.GroundFriction(mu, eps_v, self.h, self.kappa, self.dhat, self.plane_n,
                                                    self.plane_o, self.x_t)
        self.pair_friction = None
        if mu > 0 and self.body is not None:
            self.pair_friction = friction.PairFriction(mu, eps_v, self.h, self.kappa, self.dhat, self.faces,
                                                       self.edges, self.body, self.x_t)

    def velocity(self, x_new):
        """v^{t+1} of the integrator from the step's solution."""
        x_new = np.asarray(x_new, dtype=np.float64)
        if self.integrator == "ie":
            return (x_new - self.x_t) / self.h
        return (3.0 * x_new - 4.0 * self.x_t + self.x_prev) / (2.0 * self.h)

    # -- pieces -----------------------------------------------------------
    def _elements(self, fn, x, **kw):
        """fn(x, tets, vol, Dm_inv, mu, lam, **kw) over all tets, by chunks
        on self.threads threads when there are more than one."""
        if self.threads <= 1:
            return fn(x, self.tets, self.vol, self.Dm_inv, self.mu, self.lam, **kw)
        from concurrent.futures import ThreadPoolExecutor
        chunks = np.array_split(np.arange(len(self.tets)), 4 * self.threads)
        with ThreadPoolExecutor(self.threads) as ex:
            parts = list(ex.map(lambda c: fn(x, self.tets[c], self.vol[c], self.Dm_inv[c], self.mu[c],
                                             self.lam[c], **kw), chunks))
        return np.concatenate(parts)

    def distances(self, x):
        return x @ self.plane_n - self.plane_o

    def energy(self, x):
        """E(x); +inf if a tet is inverted or a vertex is on/below the plane."""
        x = np.asarray(x, dtype=np.float64)
        dx = x[self.free] - self.x_tilde[self.free]
        K = 0.5 * np.sum(self.mass[self.free] * np.sum(dx * dx, axis=1))
        Psi = np.sum(self._elements(elastic.element_energy, x))
        B = 0.0
        if self.contact:
            B = self.kappa * np.sum(barrier.b(self.distances(x), self.dhat))
        D = self.friction.energy(x) if self.friction is not None else 0.0
        if self.pair_friction is not None:
            D += self.pair_friction.energy(x)
        if self.body is not None:
            pt, ee = self.pairs(x)
            B = B + contact.pair_energy(x, self.faces, self.edges, pt, ee, self.kappa, self.dhat)
        return K + self.ah2 * (Psi + B + D)

    def pairs(self, x):
        """Mesh-mesh pairs of different bodies closer than dhat at x."""
        return contact.contact_pairs(x, self.faces, self.edges, self.body, self.dhat)

    def gradient(self, x):
        """dE/dx as [n,3]; zero on Dirichlet vertices."""
        x = np.asarray(x, dtype=np.float64)
        g = self.mass[:, None] * (x - self.x_tilde)
        ge = self._elements(elastic.element_gradient, x)
        gel = np.zeros((self.n, 3))
        np.add.at(gel, self.tets.ravel(), ge.reshape(-1, 3))
        if self.contact:
            gel += self.kappa * barrier.db(self.distances(x), self.dhat)[:, None] \
                * self.plane_n[None, :]
        if self.friction is not None:
            gel += self.friction.gradient(x)
        if self.pair_friction is not None:
            gel += self.pair_friction.gradient(x)
        if self.body is not None:
            pt, ee = self.pairs(x)
            gel += contact.pair_gradient(x, self.faces, self.edges, pt, ee, self.kappa, self.dhat)
        g += self.ah2 * gel
        g[self.pinned] = 0.0
        return g

    def hessian(self, x, elem_scale=None):
        """Projected Hessian as a (3n x 3n) CSR matrix:
        M + h^2 (sum_e c_e vol_e B^T [dP/dF]_+ B + kappa sum_v b''(d_v) n n^T),
        with Dirichlet rows and columns replaced by the identity.  c_e = 1
        unless ``elem_scale`` gives it: a cubature of the elastic term
        (Sec. 3.8) passes c_e = w_e / vol_e on its elements and 0 elsewhere;
        mass and barrier terms stay fully integrated."""
        x = np.asarray(x, dtype=np.float64)
        He = self._elements(elastic.element_hessian, x, project=self.project)
        if elem_scale is not None:
            He = He * np.asarray(elem_scale, dtype=np.float64)[:, None, None]
        dof = (3 * self.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
        rows = np.repeat(dof, 12, axis=1).ravel()
        cols = np.tile(dof, (1, 12)).ravel()
        vals = (self.ah2 * He).ravel()
        diag_idx = np.arange(3 * self.n)
        diag_val = np.repeat(self.mass, 3)
        rows = np.concatenate([rows, diag_idx])
        cols = np.concatenate([cols, diag_idx])
        vals = np.concatenate([vals, diag_val])
        if self.contact:
            k2 = self.kappa * barrier.d2b(self.distances(x), self.dhat)
            nn = np.outer(self.plane_n, self.plane_n)
            act = np.nonzero(k2)[0]
            r = (3 * act[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
            c = (3 * act[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
            rows = np.concatenate([rows, r.ravel()])
            cols = np.concatenate([cols, c.ravel()])
            vals = np.concatenate([vals, (self.ah2 * k2[act, None, None] * nn[None]).ravel()])
        if self.body is not None:
            pt, ee = self.pairs(x)
            items = [("pt", np.array([v, *self.faces[k]])) for v, k in pt]
            items += [("ee", np.array([*self.edges[i], *self.edges[j]])) for i, j in ee]
            for kind, vids in items:
                Hp = contact.pair_barrier_hessian(kind, x[vids], self.kappa, self.dhat)
                dof = (3 * vids[:, None] + np.arange(3)[None, :]).ravel()
                rows = np.concatenate([rows, np.repeat(dof, 12)])
                cols = np.concatenate([cols, np.tile(dof, 12)])
                vals = np.concatenate([vals, (self.ah2 * Hp).ravel()])
        if self.friction is not None:
            Hf = self.friction.hessian_blocks(x)
            act = np.nonzero(self.friction.lam > 0)[0]
            r = (3 * act[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
            c = (3 * act[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
            rows = np.concatenate([rows, r.ravel()])
            cols = np.concatenate([cols, c.ravel()])
            vals = np.concatenate([vals, (self.ah2 * Hf[act]).ravel()])
        if self.pair_friction is not None and len(self.pair_friction.vids):
            Hp = self.pair_friction.hessian_pairs(x)
            dof = (3 * self.pair_friction.vids[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
            rows = np.concatenate([rows, np.repeat(dof, 12, axis=1).ravel()])
            cols = np.concatenate([cols, np.tile(dof, (1, 12)).ravel()])
            vals = np.concatenate([vals, (self.ah2 * Hp).ravel()])
        H = sp.coo_matrix((vals, (rows, cols)), shape=(3 * self.n, 3 * self.n)).tocsr()
        fixed = np.repeat(self.pinned, 3)
        if fixed.any():
            keep = sp.diags((~fixed).astype(np.float64))
            H = (keep @ H @ keep + sp.diags(fixed.astype(np.float64))).tocsr()
        H.sum_duplicates()
        H.eliminate_zeros()
        return H

    def feasible(self, x):
        """True when every tet has J > 0, with contact every vertex is
        strictly above the plane, and with bodies no two of them touch."""
        F = elastic.deformation_gradient(x, self.tets, self.Dm_inv)
        if np.any(np.linalg.det(F) <= 0):
            return False
        if self.contact and np.any(self.distances(x) <= 0):
            return False
        if self.body is not None:
            pt, ee = contact.contact_pairs(x, self.faces, self.edges, self.body, 1e-300)
            if pt or ee:          # touching pairs (the CCD filter keeps them from crossing)
                return False
        return True
