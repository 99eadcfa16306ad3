"""The device arithmetic of friction between bodies checked on the CPU.

The friction kernels in contact.cu (``k_friction_lag``,
``k_friction_scatter``, ``k_friction_energy``) build each lagged pair's
frame with ``friction_frame`` and its slip and 3 x 3 block with
``friction_slip`` and ``friction_block`` (contact_geom.cuh).  The normal force
and the mollifier come from the ground friction's ``fric_lambda``,
``fric_ratio``, ``fric_slope`` and ``fric_f0`` (mls_internal.cuh).  This test
compiles those functions from their source text with g++.  A driver composes
them as the kernels do: the frame and mu lambda at x^t; at x the energy term
mu lambda f0(y), the gradient mu lambda (f1/y) w_a u and the blocks
w_a w_b mu lambda K.  The results are compared pair by pair with the
oracle's ``friction.PairFriction`` on pairs with every closest-feature kind,
at zero slip, in the sticking range and sliding.  The library's h^2 factor
and the coupling table are outside this check; the GPU tests cover them.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import contact, friction

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_13386_gb300", "csrc")
MU, EPS_V, H, KAPPA, DHAT = 0.5, 1e-3, 0.01, 1e3, 0.05
EPS = EPS_V * H

_PRELUDE = r'''
#include <cmath>
#include <cstdlib>
#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
using std::log;
using std::sqrt;
namespace mls { struct Vec4d { double x, y, z, w; }; }
'''

_DRIVER = r'''
using namespace mls;
using namespace mls::cgeom;
extern "C" void friction_pair(int kind, const double* Xt, const double* X, double mu, double kappa, double dhat,
                              double eps, double* w_out, double* n_out, double* mul_out, double* energy_out,
                              double* grad_out, double* hess_out) {
  D3 Pt[4], Px[4], dx[4];
  for (int a = 0; a < 4; ++a) {
    Pt[a] = D3{Xt[3 * a], Xt[3 * a + 1], Xt[3 * a + 2]};
    Px[a] = D3{X[3 * a], X[3 * a + 1], X[3 * a + 2]};
    dx[a] = sub(Px[a], Pt[a]);
  }
  double w[4];
  D3 n;
  const double d = friction_frame(kind, Pt, w, n);
  const double mul = mu * fric_lambda(d, dhat, kappa);
  D3 u;
  const double y = friction_slip(w, n, dx, u);
  const double ratio = fric_ratio(y, eps), slope = fric_slope(y, eps);
  double K[9];
  friction_block(n, u, y, ratio, slope, K);
  for (int a = 0; a < 4; ++a) w_out[a] = w[a];
  n_out[0] = n.x; n_out[1] = n.y; n_out[2] = n.z;
  *mul_out = mul;
  *energy_out = mul * fric_f0(y, eps);
  const double uc[3] = {u.x, u.y, u.z};
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) grad_out[3 * a + c] = mul * ratio * w[a] * uc[c];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) hess_out[(3 * a + r) * 12 + 3 * b + c] = mul * w[a] * w[b] * K[3 * r + c];
}
'''


@pytest.fixture(scope="module")
def fric(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    geom = open(os.path.join(CSRC, "contact_geom.cuh")).read().replace("#pragma once", "")
    hdr = open(os.path.join(CSRC, "mls_internal.cuh")).read()
    a = hdr.index("// ---- lagged point-plane friction")
    helpers = hdr[a:hdr.index("}  // namespace mls", a)]
    d = tmp_path_factory.mktemp("pair_friction")
    cpp, so = d / "pair_friction.cpp", d / "pair_friction.so"
    cpp.write_text(_PRELUDE + "namespace mls {\n" + helpers + "}\n" + geom + _DRIVER)
    res = subprocess.run([gxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-o", str(so), str(cpp)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    lib = C.CDLL(str(so))
    P = C.POINTER(C.c_double)
    lib.friction_pair.argtypes = [C.c_int, P, P, C.c_double, C.c_double, C.c_double, C.c_double, P, P, P, P, P, P]
    lib.friction_pair.restype = None

    def run(kind, Xt, X):
        Xt = np.ascontiguousarray(Xt, dtype=np.float64)
        X = np.ascontiguousarray(X, dtype=np.float64)
        w, n, mul, e = np.zeros(4), np.zeros(3), np.zeros(1), np.zeros(1)
        g, Hm = np.zeros(12), np.zeros(144)
        lib.friction_pair(int(kind), Xt.ctypes.data_as(P), X.ctypes.data_as(P), MU, KAPPA, DHAT, EPS,
                          *[v.ctypes.data_as(P) for v in (w, n, mul, e, g, Hm)])
        return w, n, mul[0], e[0], g.reshape(4, 3), Hm.reshape(12, 12)
    return run


def _two_tets(seed, gap=0.01):
    """Two tets of different bodies whose pairs within dhat have every
    closest-feature kind (the configuration of the oracle's friction pins)."""
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.3, 0.3, -0.5],
                  [0.2, 0.2, gap], [0.75, 0.32, gap], [0.3, 0.6, 0.6], [0.6, 0.5, 0.8]], dtype=np.float64)
    X[4:, :2] += rng.uniform(-0.01, 0.01, 2)
    X += 1e-3 * rng.normal(size=X.shape)
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    body = np.array([0, 0, 0, 0, 1, 1, 1, 1])
    faces = contact.boundary_faces(tets)
    return X, faces, contact.face_edges(faces), body


@pytest.mark.parametrize("seed", [0, 2, 3, 6])
@pytest.mark.parametrize("scale", [0.0, 0.3 * EPS, 30 * EPS])
def test_pair_friction_device_math_matches_oracle(fric, seed, scale):
    Xt, faces, edges, body = _two_tets(seed)
    pf = friction.PairFriction(MU, EPS_V, H, KAPPA, DHAT, faces, edges, body, Xt)
    assert len(pf.vids) == 6
    rng = np.random.default_rng(seed + 100)
    X = Xt + scale * rng.normal(size=Xt.shape)
    E_o, g_o, H_o = pf.energy(X), pf.gradient(X), pf.hessian_pairs(X)
    E, g = 0.0, np.zeros_like(Xt)
    gmax, hmax = np.abs(g_o).max(), np.abs(H_o).max()
    for k, vids in enumerate(pf.vids):
        kind = 0 if k < pf.n_pt else 1
        w, n, mul, e, gk, Hk = fric(kind, Xt[vids], X[vids])
        assert np.allclose(w, pf.w[k], rtol=0, atol=1e-12)
        assert np.allclose(n, pf.n[k], rtol=0, atol=1e-12)
        assert mul == pytest.approx(MU * pf.lam[k], rel=1e-12)
        E += e
        np.add.at(g, vids, gk)
        assert np.allclose(Hk, H_o[k], rtol=0, atol=1e-11 * hmax)
    assert E == pytest.approx(E_o, rel=1e-12)
    assert np.allclose(g, g_o, rtol=0, atol=1e-11 * max(gmax, 1e-300))


def test_pair_friction_device_math_ignores_normal_motion(fric):
    """A move along the pair's normal is no slip: energy at its rest value
    mu lambda eps / 3, zero gradient; the same move without the projection
    (an unprojected slip, planted in the oracle's formula here) would not be."""
    Xt, faces, edges, body = _two_tets(0)
    pf = friction.PairFriction(MU, EPS_V, H, KAPPA, DHAT, faces, edges, body, Xt)
    vids, kind = pf.vids[0], 0
    X = Xt.copy()
    X[vids[0]] += 10 * EPS * pf.n[0]
    w, n, mul, e, gk, Hk = fric(kind, Xt[vids], X[vids])
    r = np.einsum("j,jc->c", pf.w[0], X[vids] - Xt[vids])
    y_unprojected = np.linalg.norm(r)
    # the gradient is zero up to the rounding of the projection, against
    # mu lambda, the size of the gradient the unprojected slip (beyond eps,
    # f1 = 1) would give
    assert e == pytest.approx(mul * EPS / 3.0, rel=1e-12)
    assert np.abs(gk).max() <= 1e-9 * mul
    assert mul * friction.f0(y_unprojected, EPS) > 10 * e
