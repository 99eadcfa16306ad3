"""Host-side modal moment-fitting cubature (Sec. 3.8, Alg. 3).

The paper integrates the elastic part of the subspace Hessian with a
cubature: a sparse set of elements with non-negative weights.  The weights
make the integral of every degree-2 combination of the subspace basis
functions exact on each partition: the constant, each u_i and each product
u_i u_j (Sec. 3.8, modal moment fitting).  This module computes that
cubature once, untimed, like the basis itself.

Per partition P (the tet partition of the basis construction, Sec. 3.6):

1. Functions: the handles whose weight is non-zero on some element of P,
   each evaluated per element as the mean of its four vertex weights (the
   value at the barycentre, as the paper does).
2. Constraints: A[alpha, e] = prod_{i in alpha} u_i(e) over the multi-indices
   alpha of degree <= 2; targets b = A vol, the discrete integral over all of
   P's elements.
3. Alg. 3: start from n_init random elements, solve min |A_S w - b| with
   w >= 0 (Lawson-Hanson NNLS); while |A_S w - b| / |b| exceeds the tolerance
   (1e-9), add elements drawn without replacement with probability
   proportional to (A_{., k} . r)^2, r the current residual, over the
   elements not yet sampled.

Readings where the paper leaves a choice open: the "basis functions" are the
scalar handle weights phi_j (one per handle; the affine factor of each
column is a polynomial the weights multiply); n_init = min(|P|, m_P) and
each round adds min(remaining, max(4, m_P // 2)) elements, m_P the number of
constraints; a round whose probabilities are all zero draws uniformly.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize as so
import scipy.sparse as sp

DEFAULT_TOL = 1e-9


def element_weights(tets, vrow, handle, phi, n_handles):
    """u[e, j]: handle j's weight averaged over the four vertices of tet e,
    as a CSR matrix [t, m]."""
    tets = np.asarray(tets, dtype=np.int64)
    vrow = np.asarray(vrow, dtype=np.int64)
    n = len(vrow) - 1
    Phi = sp.csr_matrix((np.asarray(phi, dtype=np.float64), np.asarray(handle, dtype=np.int64), vrow),
                        shape=(n, n_handles))
    t = len(tets)
    avg = sp.csr_matrix((np.full(4 * t, 0.25), tets.ravel(), np.arange(0, 4 * t + 1, 4)), shape=(t, n))
    return (avg @ Phi).tocsr()


def moment_matrix(Ue):
    """Rows 1, u_i, u_i u_j (i <= j) of a dense [n_elem, k] block of element
    weights: the constraint matrix A [m, n_elem] of modal moment fitting."""
    n, k = Ue.shape
    rows = [np.ones((1, n)), Ue.T]
    iu, ju = np.triu_indices(k)
    rows.append((Ue[:, iu] * Ue[:, ju]).T)
    return np.concatenate(rows, axis=0)


def _fit(A, b, rng, tol):
    """Alg. 3 on one partition: returns (local element indices, weights)."""
    m, n = A.shape
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    n_init = min(n, m)
    n_add = max(4, m // 2)
    S = np.sort(rng.choice(n, size=n_init, replace=False))
    while True:
        w, _ = so.nnls(A[:, S], b, maxiter=50 * max(len(S), 1))
        r = A[:, S] @ w - b
        if np.linalg.norm(r) <= tol * bn or len(S) == n:
            break
        cand = np.setdiff1d(np.arange(n), S, assume_unique=True)
        rho = (A[:, cand].T @ r) ** 2
        k = min(len(cand), n_add)
        pos = np.count_nonzero(rho)
        if pos >= k and rho.sum() > 0:
            pick = rng.choice(cand, size=k, replace=False, p=rho / rho.sum())
        else:
            pick = rng.choice(cand, size=k, replace=False)
        S = np.sort(np.concatenate([S, pick]))
    keep = w > 0
    return S[keep], w[keep]


def _partition_job(args):
    A, b, seed, tol = args
    return _fit(A, b, np.random.default_rng(seed), tol)


def build_cubature(X, tets, basis, tol=DEFAULT_TOL, seed=0, workers=None):
    """Cubature of the elastic energy for an SMS basis (dict from
    ``basis.build_sms_basis``, or any dict with ``vrow``/``handle``/``phi``,
    ``origins`` and a per-tet ``partition``).  Returns a dict:

    * ``elem`` int32 [c]: cubature elements (tet indices), sorted;
    * ``weight`` float64 [c]: their weights (volumes, > 0);
    * ``scale`` float64 [t]: weight / rest volume per tet, 0 off the cubature
      (the factor on each element Hessian);
    * ``residual`` float64 [p]: |A w - b| / |b| per partition;
    * ``constraints`` int [p], ``points`` int [p]: m_P and the points kept.
    """
    from .basis import _rest

    X = np.asarray(X, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    part = np.asarray(basis["partition"], dtype=np.int64)
    m = len(basis["origins"])
    vol, _ = _rest(X, tets)
    U = element_weights(tets, basis["vrow"], basis["handle"], basis["phi"], m)
    jobs, members = [], []
    for P in range(int(part.max()) + 1):
        el = np.nonzero(part == P)[0]
        members.append(el)
        sub = U[el]
        funcs = np.unique(sub.indices)
        Ue = sub[:, funcs].toarray()
        A = moment_matrix(Ue)
        b = A @ vol[el]
        jobs.append((A, b, seed * 1_000_003 + P, tol))
    if workers is None:
        import os
        workers = min(16, os.cpu_count() or 1) if len(jobs) >= 32 else 1
    if workers <= 1:
        fits = [_partition_job(j) for j in jobs]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            fits = pool.map(_partition_job, jobs, chunksize=max(1, len(jobs) // (4 * workers)))
    elem, weight, res, cons, pts = [], [], [], [], []
    for (A, b, _, _), el, (S, w) in zip(jobs, members, fits):
        elem.append(el[S])
        weight.append(w)
        full = np.zeros(len(el))
        full[S] = w
        res.append(float(np.linalg.norm(A @ full - b) / max(np.linalg.norm(b), 1e-300)))
        cons.append(A.shape[0])
        pts.append(len(S))
    elem = np.concatenate(elem)
    weight = np.concatenate(weight)
    order = np.argsort(elem)
    elem, weight = elem[order], weight[order]
    scale = np.zeros(len(tets))
    scale[elem] = weight / vol[elem]
    return {"elem": elem.astype(np.int32), "weight": weight, "scale": scale, "residual": np.asarray(res),
            "constraints": np.asarray(cons), "points": np.asarray(pts)}
