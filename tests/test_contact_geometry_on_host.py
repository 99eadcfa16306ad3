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
#include <cstdlib>
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
// test-only: serial cyclic Jacobi projection of the symmetric k x k A (ld 12) to the PSD cone
static void jacobi_psd(double* A, int k) {
  double V[144];
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) V[i * 12 + j] = i == j;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = i + 1; j < k; ++j) off += A[i * 12 + j] * A[i * 12 + j];
    if (off < 1e-300) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[p * 12 + q];
        if (apq == 0.0) continue;
        const double tau = (A[q * 12 + q] - A[p * 12 + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        for (int r = 0; r < k; ++r) {
          const double a = A[r * 12 + p], b = A[r * 12 + q];
          A[r * 12 + p] = c * a - sn * b; A[r * 12 + q] = sn * a + c * b;
        }
        for (int r = 0; r < k; ++r) {
          const double a = A[p * 12 + r], b = A[q * 12 + r];
          A[p * 12 + r] = c * a - sn * b; A[q * 12 + r] = sn * a + c * b;
        }
        for (int r = 0; r < k; ++r) {
          const double a = V[r * 12 + p], b = V[r * 12 + q];
          V[r * 12 + p] = c * a - sn * b; V[r * 12 + q] = sn * a + c * b;
        }
      }
  }
  double lam[12];
  for (int i = 0; i < k; ++i) lam[i] = A[i * 12 + i] > 0 ? A[i * 12 + i] : 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int m = 0; m < k; ++m) s += V[i * 12 + m] * lam[m] * V[j * 12 + m];
      A[i * 12 + j] = s;
    }
}
// the barrier Hessian of a pair through the reduced edge-vector space, as the pair kernel forms it
extern "C" void projected(int kind, const double* X, double kappa, double dhat, double* Hb, double* g) {
  D3 P[4];
  load(X, P);
  const Feature F = kind == 0 ? pt_feature(P[0], P[1], P[2], P[3]) : ee_feature(P[0], P[1], P[2], P[3]);
  Reduced Rd;
  feature_reduced(F, P, Rd);
  const double d = Rd.d, r = d - dhat;
  const double b1 = d < dhat ? kappa * (-2.0 * r * std::log(d / dhat) - r * r / d) : 0.0;
  const double b2 = d < dhat ? kappa * (-2.0 * std::log(d / dhat) - 4.0 * r / d + r * r / (d * d)) : 0.0;
  const int ny = 3 * Rd.nb;
  double N[144];
  for (int a = 0; a < ny; ++a)
    for (int b = 0; b < ny; ++b) N[a * 12 + b] = reduced_entry(Rd, b1, b2, a, b);
  jacobi_psd(N, ny);
  for (int q = 0; q < 144; ++q) Hb[q] = 0.0;
  for (int q = 0; q < 12; ++q) g[q] = 0.0;
  for (int v = 0; v < F.nv; ++v)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < Rd.nb; ++k) s += Rd.C[k][v] * Rd.gdy[3 * k + c];
      g[3 * F.idx[v] + c] = b1 * s;
      for (int w = 0; w < F.nv; ++w)
        for (int e = 0; e < 3; ++e) Hb[(3 * F.idx[v] + c) * 12 + 3 * F.idx[w] + e] = reduced_back(Rd, N, 12, v, c, w, e);
    }
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
    lib.projected.argtypes = [C.c_int, P, C.c_double, C.c_double, P, P]
    lib.projected.restype = None
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


def test_reduced_space_projection_matches_oracle(geom):
    """The pair kernel projects the barrier Hessian in the feature's edge-
    vector space (N = R M R^T of order 3 nb) and maps it back with Q; this
    must equal the oracle's projection of the full 12 x 12 pair Hessian
    (1e-9 of its largest entry), and the gradient kappa b' grad d (1e-10)."""
    from oracle import barrier
    kind, X = _pairs()
    P = C.POINTER(C.c_double)
    dhat, kappa = 10.0, 3.0
    for k, x in zip(kind, X):
        x = np.ascontiguousarray(x, dtype=np.float64)
        kk = "pt" if k == 0 else "ee"
        Hb, g = np.zeros(144), np.zeros(12)
        geom.projected(int(k), x.ctypes.data_as(P), kappa, dhat, Hb.ctypes.data_as(P), g.ctypes.data_as(P))
        Hb_o = contact.pair_barrier_hessian(kk, x, kappa, dhat)
        assert np.max(np.abs(Hb.reshape(12, 12) - Hb_o)) <= 1e-9 * np.max(np.abs(Hb_o))
        d_o, g_o, _ = contact.pair_distance_derivatives(kk, x)
        g_ref = kappa * barrier.db(np.array([d_o]), dhat)[0] * g_o
        assert np.max(np.abs(g - g_ref)) <= 1e-10 * np.max(np.abs(g_ref))
