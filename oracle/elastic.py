"""Non-inverting Neo-Hookean elasticity on linear tetrahedra (oracle).

The paper states only that every simulation uses a non-inverting Neo-Hookean
model (Sec. 4, Results).  The reading used throughout this project:

    psi(F) = mu/2 (tr(F^T F) - 3) - mu ln J + lam/2 (ln J)^2,   J = det F > 0,
    psi(F) = +inf for J <= 0,
    mu = E / (2 (1 + nu)),  lam = E nu / ((1 + nu)(1 - 2 nu)).

F is the deformation gradient of a linear tet, F = D_s D_m^{-1} with
D_s = [x1-x0, x2-x0, x3-x0] and D_m the same for the rest positions.  The
element energy is vol * psi(F).

Flattening conventions used by every oracle function:
  vec(F)[3a + b] = F[a, b]   (row-major 3x3)
  element DOF   3 j + c      (vertex j in 0..3 of the tet, coordinate c)

The element Hessian is vol * B^T [dP/dF]_+ B, where B = dvec(F)/dx (9 x 12)
and [.]_+ replaces the negative eigenvalues of the symmetric 9x9 stress
derivative by zero (projection onto the PSD cone).  The paper does not state
its projection; this per-element PSD clamp of the 9x9 is the reading used.
"""
from __future__ import annotations

import numpy as np


def lame(E, nu):
    """Lame parameters (mu, lam) from Young's modulus and Poisson ratio."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def edge_matrix(x, tets):
    """D = [x1-x0, x2-x0, x3-x0] as columns, one 3x3 per tet: [t,3,3]."""
    x = np.asarray(x, dtype=np.float64)
    T = np.asarray(tets)
    return np.stack([x[T[:, 1]] - x[T[:, 0]], x[T[:, 2]] - x[T[:, 0]],
                     x[T[:, 3]] - x[T[:, 0]]], axis=-1)


def rest_shape(X, tets):
    """Rest volume and D_m^{-1} per tet.  Raises if a tet is not positively
    oriented at rest."""
    Dm = edge_matrix(X, tets)
    det = np.linalg.det(Dm)
    if np.any(det <= 0):
        raise ValueError("tet with non-positive rest volume")
    return det / 6.0, np.linalg.inv(Dm)


def deformation_gradient(x, tets, Dm_inv):
    """F = D_s D_m^{-1} per tet: [t,3,3]."""
    return edge_matrix(x, tets) @ Dm_inv


def psi(F, mu, lam):
    """Energy density; +inf where det F <= 0 (the model is non-inverting)."""
    F = np.asarray(F, dtype=np.float64)
    J = np.linalg.det(F)
    out = np.full(J.shape, np.inf)
    ok = J > 0
    I2 = np.einsum("...ab,...ab->...", F, F)
    lnJ = np.log(np.where(ok, J, 1.0))
    mu = np.broadcast_to(mu, J.shape)
    lam = np.broadcast_to(lam, J.shape)
    val = 0.5 * mu * (I2 - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2
    out[ok] = val[ok]
    return out


def first_pk(F, mu, lam):
    """P = dpsi/dF = mu (F - F^{-T}) + lam ln J F^{-T}   [t,3,3]."""
    F = np.asarray(F, dtype=np.float64)
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(J)
    mu = np.asarray(mu)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    return mu * (F - FinvT) + lam * lnJ[..., None, None] * FinvT


def stress_derivative(F, mu, lam):
    """dP/dF as a 9x9 matrix per tet, rows vec(P) and columns vec(F).

    Differentiating P = mu F + (lam ln J - mu) F^{-T} with d ln J = F^{-T} : dF
    and d(F^{-T}) = -F^{-T} dF^T F^{-T}:
      dP_ij/dF_kl = mu d_ik d_jl + lam G_ij G_kl - (lam ln J - mu) G_il G_kj,
    with G = F^{-T}.
    """
    F = np.asarray(F, dtype=np.float64)
    G = np.swapaxes(np.linalg.inv(F), -1, -2)
    lnJ = np.log(np.linalg.det(F))
    mu = np.asarray(mu, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    eye = np.eye(3)
    T1 = np.einsum("ik,jl->ijkl", eye, eye)
    T1 = np.broadcast_to(T1, F.shape[:-2] + (3, 3, 3, 3))
    T2 = np.einsum("...ij,...kl->...ijkl", G, G)
    T3 = np.einsum("...il,...kj->...ijkl", G, G)
    c3 = lam * lnJ - mu
    D = (mu[..., None, None, None, None] * T1 + lam[..., None, None, None, None] * T2
         - c3[..., None, None, None, None] * T3)
    return D.reshape(F.shape[:-2] + (9, 9))


def dF_dx(Dm_inv):
    """B = d vec(F) / d x_e as [t,9,12].

    With F_ab = sum_k (x_{k+1,a} - x_{0,a}) Dm_inv[k,b]:
      dF_ab/dx_{j,c} = d_ac Dm_inv[j-1, b]            for j = 1, 2, 3,
      dF_ab/dx_{0,c} = -d_ac sum_k Dm_inv[k, b].
    """
    Dm_inv = np.asarray(Dm_inv, dtype=np.float64)
    t = Dm_inv.shape[0]
    B = np.zeros((t, 9, 12))
    for a in range(3):
        for b in range(3):
            row = 3 * a + b
            for j in range(1, 4):
                B[:, row, 3 * j + a] = Dm_inv[:, j - 1, b]
            B[:, row, a] = -Dm_inv[:, :, b].sum(axis=1)
    return B


def psd_project(A):
    """Closest PSD matrix in the Frobenius norm: eigenvalues below zero
    clamped to zero (library eigh on each symmetric matrix)."""
    A = 0.5 * (A + np.swapaxes(A, -1, -2))
    w, V = np.linalg.eigh(A)
    w = np.maximum(w, 0.0)
    return (V * w[..., None, :]) @ np.swapaxes(V, -1, -2)


def element_energy(x, tets, vol, Dm_inv, mu, lam):
    """vol_e * psi(F_e) per tet (+inf for inverted tets)."""
    return vol * psi(deformation_gradient(x, tets, Dm_inv), mu, lam)


def element_gradient(x, tets, vol, Dm_inv, mu, lam):
    """d(vol psi)/dx_e = vol B^T vec(P), [t,12]."""
    F = deformation_gradient(x, tets, Dm_inv)
    P = first_pk(F, mu, lam).reshape(-1, 9)
    B = dF_dx(Dm_inv)
    return vol[:, None] * np.einsum("tri,tr->ti", B, P)


def element_hessian(x, tets, vol, Dm_inv, mu, lam, project=True):
    """vol B^T [dP/dF]_(+) B, [t,12,12]; the 9x9 is PSD-projected when
    ``project`` is true."""
    F = deformation_gradient(x, tets, Dm_inv)
    D = stress_derivative(F, mu, lam)
    if project:
        D = psd_project(D)
    B = dF_dx(Dm_inv)
    return vol[:, None, None] * np.einsum("tri,trs,tsj->tij", B, D, B)
