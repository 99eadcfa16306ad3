"""Point-plane IPC log barrier (oracle).

The paper's contact term B in Eq. IP is the IPC barrier, cited but not
written out.  The reading used throughout this project, for a vertex at
unsquared distance d = n . x - o above the plane:

    b(d) = -(d - dhat)^2 ln(d / dhat)   for 0 < d < dhat,
    b(d) = 0                            for d >= dhat,
    b(d) = +inf                         for d <= 0,

and B(x) = kappa * sum_v b(d_v), entering E with the same h^2 factor as the
elastic energy.  Its gradient with respect to x_v is kappa b'(d) n and its
Hessian kappa b''(d) n n^T, positive semi-definite because b'' > 0 on
(0, dhat).
"""
from __future__ import annotations

import numpy as np


def b(d, dhat):
    """Barrier value at distance ``d``."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    act = (d > 0) & (d < dhat)
    dd = d[act]
    out[act] = -((dd - dhat) ** 2) * np.log(dd / dhat)
    out[d <= 0] = np.inf
    return out


def db(d, dhat):
    """b'(d) = -2 (d - dhat) ln(d/dhat) - (d - dhat)^2 / d on (0, dhat)."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    act = (d > 0) & (d < dhat)
    dd = d[act]
    out[act] = -2.0 * (dd - dhat) * np.log(dd / dhat) - (dd - dhat) ** 2 / dd
    return out


def d2b(d, dhat):
    """b''(d) = -2 ln(d/dhat) - 4 (d - dhat)/d + (d - dhat)^2 / d^2 on (0, dhat)."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    act = (d > 0) & (d < dhat)
    dd = d[act]
    out[act] = (-2.0 * np.log(dd / dhat) - 4.0 * (dd - dhat) / dd
                + (dd - dhat) ** 2 / dd ** 2)
    return out
