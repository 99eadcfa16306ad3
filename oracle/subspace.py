"""Subspace bases and the multilevel preconditioner algebra (oracle).

LBS basis (Eq. LBS, Sec. 3.4-3.5).  For handle j with origin o_j and scalar
weight phi_j(v) at vertex v, the 3x12 block of U at (v, j) is
phi_j(v) P(X_v - o_j) with P(y) = I_3 (x) [1, y_x, y_y, y_z], i.e.

    U[3 v + c, 12 j + 4 c + l] = phi_j(v) * a_l,   a = [1, X_v - o_j],

so q_j in R^12 is the row-major flattening of a 3x4 affine matrix.  The SMS
basis has compactly supported weights (Sec. 3.5); the affine basis has one
handle per object at its centre of mass with phi = 1 (Sec. 3.4).

Coarse operators are Galerkin products U^T H U (the "subspace sandwich
matrices" of Alg. 2 / Sec. 3.7.1), here formed explicitly.

Two-level preconditioners, applied to a residual r with S = omega D^{-1}
(D = 3x3 block diagonal of H) and Q = U A_c^{-1} U^T:
  additive        z = S r + Q r
  multiplicative  z1 = S r;  z2 = z1 + Q (r - H z1);  z = z2 + S (r - H z2)
The multiplicative form mirrors the paper's ordering inside one Newton
iteration (subspace correction, then full-space Jacobi refinement) and is
symmetric; it is positive definite when omega * lambda_max(D^{-1} H) < 2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def lbs_basis_matrix(X, origins, vrow, handle, phi):
    """Sparse U (3n x 12m) from per-vertex CSR weights (vrow, handle, phi)."""
    X = np.asarray(X, dtype=np.float64)
    origins = np.asarray(origins, dtype=np.float64)
    n = X.shape[0]
    m = origins.shape[0]
    rows, cols, vals = [], [], []
    for v in range(n):
        for s in range(vrow[v], vrow[v + 1]):
            j = int(handle[s])
            a = np.concatenate([[1.0], X[v] - origins[j]])
            for c in range(3):
                for l in range(4):
                    rows.append(3 * v + c)
                    cols.append(12 * j + 4 * c + l)
                    vals.append(phi[s] * a[l])
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * n, 12 * m))


def affine_basis_matrix(X, object_id=None, mass=None):
    """Per-object affine basis: one handle per object at its (mass-weighted)
    centre with phi = 1 on every vertex of the object (Sec. 3.4)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    obj = np.zeros(n, dtype=np.int64) if object_id is None else np.asarray(object_id)
    w = np.ones(n) if mass is None else np.asarray(mass, dtype=np.float64)
    n_obj = int(obj.max()) + 1
    origins = np.zeros((n_obj, 3))
    for o in range(n_obj):
        sel = obj == o
        origins[o] = (w[sel, None] * X[sel]).sum(0) / w[sel].sum()
    vrow = np.arange(n + 1)
    return origins, lbs_basis_matrix(X, origins, vrow, obj, np.ones(n))


def prolong(U, q):
    """w = U q (lift to full space), returned as [n,3]."""
    return (U @ np.asarray(q, dtype=np.float64).ravel()).reshape(-1, 3)


def restrict(U, r):
    """z = U^T r (restriction to the subspace), returned as [m,12]."""
    return (U.T @ np.asarray(r, dtype=np.float64).ravel()).reshape(-1, 12)


def galerkin(H, U):
    """Dense U^T H U."""
    return np.asarray((U.T @ (H @ U)).todense())


def block_diagonal_inverse(H):
    """D^{-1} for the 3x3 block diagonal D of H, as a sparse matrix."""
    n3 = H.shape[0]
    Hd = H.tocsr()
    blocks = np.zeros((n3 // 3, 3, 3))
    for v in range(n3 // 3):
        blocks[v] = Hd[3 * v:3 * v + 3, 3 * v:3 * v + 3].toarray()
    inv = np.linalg.inv(blocks)
    return sp.csr_matrix(sp.block_diag([sp.coo_matrix(b) for b in inv], format="csr"))


def coarse_solve(Ac, rhs):
    """A_c^{-1} rhs by a library Cholesky factorisation."""
    L = np.linalg.cholesky(Ac)
    y = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.T, y)


def two_level_apply(H, U, Ac, r, mode="multiplicative", omega=1.0, Dinv=None):
    """Apply the two-level preconditioner defined in the module docstring."""
    r = np.asarray(r, dtype=np.float64).ravel()
    if Dinv is None:
        Dinv = block_diagonal_inverse(H)

    def S(v):
        return omega * (Dinv @ v)

    def Q(v):
        return U @ coarse_solve(Ac, U.T @ v)

    if mode == "additive":
        return S(r) + Q(r)
    if mode == "multiplicative":
        z1 = S(r)
        z2 = z1 + Q(r - H @ z1)
        return z2 + S(r - H @ z2)
    if mode == "coarse":
        return Q(r)
    raise ValueError(mode)


def paper_direction(H, g, U, n_cg):
    """One direction of the paper's inexact Newton iteration (Alg. 1,
    Alg. 2), with the two subspace levels solved exactly: the affine level
    lies in span U (the SMS basis reproduces affine motions, Sec. 3.5), so
    an exact solve in span U already contains it.

        d_s = U (U^T H U)^{-1} U^T (-g)                 (subspace direction)
        d_f = n_cg iterations of block-Jacobi PCG on H d_f = -g - H d_s,
              started from d_f = 0                       (full-space refinement)

    Returns (d_s, d_f) as flat arrays.  Test infrastructure only."""
    from . import pcg as opcg
    g = np.asarray(g, dtype=np.float64).ravel()
    Ac = galerkin(H, U)
    ds = U @ coarse_solve(Ac, U.T @ (-g))
    r = -g - H @ ds
    Dinv = block_diagonal_inverse(H)
    # (stops early only at a relative residual of 1e-14, where a fixed
    # iteration count has nothing left to do)
    df, _ = opcg.pcg(lambda v: H @ v, r, lambda v: Dinv @ v, rtol=1e-14, max_iter=n_cg)
    return np.asarray(ds).ravel(), df


def handle_block_jacobi(A, block=12):
    """Inverse of the 12 x 12 diagonal blocks of a subspace matrix, the
    preconditioner of the subspace PCG solves (Sec. 3.7.1: one block per
    handle's degrees of freedom), as a function v -> D^{-1} v."""
    A = sp.csr_matrix(A) if sp.issparse(A) else sp.csr_matrix(np.asarray(A))
    r = A.shape[0]
    inv = [np.linalg.inv(A[k:k + block, k:k + block].toarray()) for k in range(0, r, block)]

    def apply(v):
        v = np.asarray(v, dtype=np.float64)
        return np.concatenate([Bi @ v[k * block:(k + 1) * block] for k, Bi in enumerate(inv)])
    return apply


def subspace_direction_literal(H, g, Ua, Us, rtol=1e-4):
    """SolveSubspaceDirection of Alg. 2 as printed, both levels by PCG:

        (Ua^T H Ua) q_a = Ua^T (-g)        PCG, 12 x 12 block Jacobi, to rtol
        d_s = Ua q_a;  r = -g - H d_s
        (Us^T H Us) q_s = Us^T r           PCG, 12 x 12 block Jacobi, to rtol
        d_s = d_s + Us q_s

    The subspace products are matrix-free, U^T (H (U q)) (Sec. 3.7.1).
    (The printed algorithm writes g for the right-hand side; the direction
    of descent takes -g.)  Returns (d_s flat, (iters_a, iters_s))."""
    from . import pcg as opcg
    g = np.asarray(g, dtype=np.float64).ravel()
    out_iters = []
    ds = np.zeros_like(g)
    r = -g
    for U in (Ua, Us):
        A_blocks = galerkin(H, U)               # only its diagonal blocks are used, as the preconditioner
        Minv = handle_block_jacobi(A_blocks)
        q, info = opcg.pcg(lambda v: U.T @ (H @ (U @ v)), U.T @ r, Minv, rtol=rtol, max_iter=100000)
        ds = ds + U @ q
        r = -g - H @ ds
        out_iters.append(info["iters"])
    return ds, tuple(out_iters)
