"""The contact kernels' geometry checked on the CPU against the oracle.

``contact_geom.cuh`` holds the device functions the mesh-mesh contact
kernels use for a primitive pair: the closest points of a point and a
triangle or of two segments, the closest feature, and the distance's
gradient and Hessian from that feature's squared-distance formula.  They
are plain double-precision arithmetic.  This test compiles the header as
host C++ with g++ (the CUDA qualifiers defined away) and compares, pair by
pair, with ``oracle/contact.py``:

* the distance of the closed primitives (1e-12 relative);
* the closest feature, its type and vertices (identical);
* grad d (1e-10) and Hess d (1e-9 of the largest entry), against the
  oracle's hyper-dual derivatives of the same feature's formula.

The GPU tests (``test_gpu_contact.py``) check the same functions through the
library on a GPU; this test needs no GPU.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import contact

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_13386_gb300", "csrc")

_PRELUDE = r'''
#include <cmath>
#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
'''

_DRIVER = r'''
using namespace mls::cgeom;
static void load(const double* X, D3 (&P)[4]) {
  for (int a = 0; a < 4; ++a) P[a] = D3{X[3 * a], X[3 * a + 1], X[3 * a + 2]};
}
extern "C" double distance(int kind, const double* X) {
  D3 P[4];
  load(X, P);
  return pair_distance(kind, P);
}
extern "C" double derivatives(int kind, const double* X, int* form_idx, double* gd, double* Hd) {
  D3 P[4];
  load(X, P);
  const Feature F = kind == 0 ? pt_feature(P[0], P[1], P[2], P[3]) : ee_feature(P[0], P[1], P[2], P[3]);
  form_idx[0] = F.form;
  form_idx[1] = F.nv;
  for (int k = 0; k < 4; ++k) form_idx[2 + k] = F.idx[k];
  return feature_derivatives(F, P, gd, Hd);
}
'''


@pytest.fixture(scope="module")
def geom(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = open(os.path.join(CSRC, "contact_geom.cuh")).read().replace("#pragma once", "")
    d = tmp_path_factory.mktemp("cgeom")
    cpp = d / "cgeom.cpp"
    cpp.write_text(_PRELUDE + src + _DRIVER)
    so = d / "cgeom.so"
    subprocess.run([gxx, "-O2", "-fPIC", "-shared", "-o", str(so), str(cpp)], check=True, capture_output=True)
    lib = C.CDLL(str(so))
    P = C.POINTER(C.c_double)
    lib.distance.argtypes = [C.c_int, P]
    lib.distance.restype = C.c_double
    lib.derivatives.argtypes = [C.c_int, P, C.POINTER(C.c_int), P, P]
    lib.derivatives.restype = C.c_double
    return lib


def _pairs(count=300, seed=13):
    r = np.random.default_rng(seed)
    X = list(r.normal(size=(count, 4, 3)))
    kind = list(r.integers(0, 2, size=count))
    for _ in range(40):  # interior features: a point over a triangle, crossing edges
        a, b, c = r.normal(size=(3, 3))
        w = r.dirichlet(np.ones(3))
        n = np.cross(b - a, c - a)
        X.append(np.array([w @ np.array([a, b, c]) + r.normal() * n / np.linalg.norm(n), a, b, c]))
        kind.append(0)
        p0, p1 = r.normal(size=(2, 3))
        m = 0.5 * (p0 + p1) + 0.3 * r.normal(size=3)
        u = r.normal(size=3)
        X.append(np.array([p0, p1, m - u, m + u]))
        kind.append(1)
    return np.array(kind), np.array(X)


_FORM = {0: "pp", 1: "pe", 2: "pt", 3: "ee"}


def test_contact_geometry_matches_oracle(geom):
    kind, X = _pairs()
    P = C.POINTER(C.c_double)
    seen = set()
    for k, x in zip(kind, X):
        x = np.ascontiguousarray(x, dtype=np.float64)
        kk = "pt" if k == 0 else "ee"
        d_ref = contact.point_triangle_distance(*x) if k == 0 else contact.edge_edge_distance(*x)
        assert geom.distance(int(k), x.ctypes.data_as(P)) == pytest.approx(d_ref, rel=1e-12)
        fi = (C.c_int * 6)()
        gd = np.zeros(12)
        Hd = np.zeros(144)
        d = geom.derivatives(int(k), x.ctypes.data_as(P), fi, gd.ctypes.data_as(P), Hd.ctypes.data_as(P))
        # the feature: type and vertices as the oracle classifies them
        t = contact._pt_type(*x) if k == 0 else contact._ee_type(*x)
        form, nv, idx = fi[0], fi[1], list(fi[2:2 + fi[1]])
        seen.add((kk, t[0]))
        if k == 0:
            want = {"pt": (2, [0, 1, 2, 3]), "pe": (1, [0, 1 + t[1], 1 + t[2]]) if t[0] == "pe" else None,
                    "pp": (0, [0, 1 + t[1]]) if t[0] == "pp" else None}[t[0]]
        else:
            want = {"ee": (3, [0, 1, 2, 3]), "pe": (1, list(t[1:])) if t[0] == "pe" else None,
                    "pp": (0, list(t[1:])) if t[0] == "pp" else None}[t[0]]
        assert (form, idx) == want, (kk, t, form, idx)
        d_o, g_o, H_o = contact.pair_distance_derivatives(kk, x)
        assert d == pytest.approx(d_o, rel=1e-12)
        assert np.max(np.abs(gd - g_o)) <= 1e-10 * np.max(np.abs(g_o))
        assert np.max(np.abs(Hd.reshape(12, 12) - H_o)) <= 1e-9 * np.max(np.abs(H_o))
    assert seen == {("pt", "pt"), ("pt", "pe"), ("pt", "pp"), ("ee", "ee"), ("ee", "pe"), ("ee", "pp")}


def test_planted_sign_error_is_caught(geom, tmp_path):
    """A dropped term in the plane form (the Hessian of m) must fail the
    comparison: the test is sensitive to the formulas, not only to d."""
    gxx = shutil.which("g++")
    src = open(os.path.join(CSRC, "contact_geom.cuh")).read().replace("#pragma once", "")
    broken = src.replace("add_skew(H, 9, 3, 6, n, -2.0 * c_hm);", "", 1)
    assert broken != src
    cpp = tmp_path / "broken.cpp"
    cpp.write_text(_PRELUDE + broken + _DRIVER)
    so = tmp_path / "broken.so"
    subprocess.run([gxx, "-O2", "-fPIC", "-shared", "-o", str(so), str(cpp)], check=True, capture_output=True)
    lib = C.CDLL(str(so))
    P = C.POINTER(C.c_double)
    lib.derivatives.argtypes = [C.c_int, P, C.POINTER(C.c_int), P, P]
    lib.derivatives.restype = C.c_double
    kind, X = _pairs()
    worst = 0.0
    for k, x in zip(kind, X):
        x = np.ascontiguousarray(x, dtype=np.float64)
        fi = (C.c_int * 6)()
        gd, Hd = np.zeros(12), np.zeros(144)
        lib.derivatives(int(k), x.ctypes.data_as(P), fi, gd.ctypes.data_as(P), Hd.ctypes.data_as(P))
        _, _, H_o = contact.pair_distance_derivatives("pt" if k == 0 else "ee", x)
        worst = max(worst, np.max(np.abs(Hd.reshape(12, 12) - H_o)) / np.max(np.abs(H_o)))
    assert worst > 1e-6
