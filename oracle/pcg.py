"""Preconditioned conjugate gradient from its textbook definition (oracle).

Solves A x = b for SPD A with an SPD preconditioner M^{-1}, starting from
x0 (default zero), and stops when |r|_2 <= rtol |b|_2.  This is the method the
paper applies at every level (Alg. 2, Sec. 3.7); here it is written once,
plainly, with float64 vectors and dot products.
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, b, apply_Minv, rtol=1e-10, max_iter=10000, x0=None):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    bnorm = float(np.linalg.norm(b))
    info = {"iters": 0, "converged": False, "rnorm": [float(np.linalg.norm(r))]}
    if bnorm == 0.0:
        info["converged"] = True
        return x, info
    z = apply_Minv(r)
    p = z.copy()
    rz = float(r @ z)
    for k in range(max_iter):
        if info["rnorm"][-1] <= rtol * bnorm:
            info["converged"] = True
            break
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        info["rnorm"].append(float(np.linalg.norm(r)))
        info["iters"] = k + 1
        z = apply_Minv(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    else:
        info["converged"] = info["rnorm"][-1] <= rtol * bnorm
    return x, info
