"""Kernel arithmetic checked on the CPU: friction terms and the BDF2 predictor.

The lagged point-plane friction term (Eq. IP, term D) enters three kernels:
the gradient gather (``k_gather_grad``), the diagonal Hessian blocks
(``k_assemble``) and the line-search energies (``k_energy``, and
``k_benergy`` of the batched path).  Their friction
branches and the helpers they call are plain double-precision arithmetic.
This test takes their exact source text from the ``.cu`` files, compiles it
as host C++ with g++, and compares the per-vertex results with the oracle's
``friction.GroundFriction``.  The GPU parity tests check the same terms
through the library on a GPU; this test needs no GPU.

The helpers are taken from the friction section of ``mls_internal.cuh``.  The
branches are the balanced blocks opened by the friction guards in the kernels.
Tolerances: with the ground plane z = 0, the plane distance is exact on both
sides, and the terms agree to rounding (1e-14 of the largest entry).  On a
tilted plane, the distance n . x - o loses digits to cancellation when it is
small, and the normal force grows like 1/d.  With d >= 1e-4 m and positions
of order 1 m, 1e-11 covers that.

The BDF2 predictor kernel (``k_predictor_bdf2``, one thread per vertex) is
checked the same way: its body runs in a loop over the vertices and must
reproduce the oracle's BDF2 predictor (Sec. 3.1) to rounding.
"""
import ctypes as C
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import friction

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_13386_gb300", "csrc")


def _block(src, pattern, nth):
    """Source text of the balanced { } block opened after the nth match of pattern."""
    starts = [m.start() for m in re.finditer(re.escape(pattern), src)]
    i = src.index("{", starts[nth])
    depth = 0
    for j in range(i, len(src)):
        if src[j] == "{":
            depth += 1
        elif src[j] == "}":
            depth -= 1
            if depth == 0:
                return src[i:j + 1]
    raise ValueError(f"unbalanced block after {pattern!r}")


_PRELUDE = r'''
#include <cmath>
#include <cstdint>
#include <vector>
using std::log;
using std::sqrt;
struct Vec4d { double x, y, z, w; };
'''

# in: plane (n, o), dhat, kappa, mu, eps, h^2 and x^t, as the kernels' parameter structs hold them
_DRIVER = r'''
struct In { double pn0, pn1, pn2, po, dhat, kappa, fmu, feps, h2; const Vec4d* xt; };
static std::vector<Vec4d> pack(int n, const double* a) {
  std::vector<Vec4d> v(n);
  for (int i = 0; i < n; ++i) v[i] = Vec4d{a[3 * i], a[3 * i + 1], a[3 * i + 2], 0.0};
  return v;
}
#define SETUP                                                                         \
  std::vector<Vec4d> X = pack(n, xs), XT = pack(n, xts);                              \
  In in{P[0], P[1], P[2], P[3], P[4], P[5], P[6], P[7], P[8], XT.data()};
extern "C" void grad_terms(int n, const double* xs, const double* xts, const double* P, double* out) {
  SETUP
  for (int v = 0; v < n; ++v) {
    const Vec4d xv = X[v];
    double sx = 0, sy = 0, sz = 0;
    GRAD_BRANCH
    out[3 * v] = sx; out[3 * v + 1] = sy; out[3 * v + 2] = sz;
  }
}
extern "C" void block_terms(int n, const double* xs, const double* xts, const double* P, double* out) {
  SETUP
  typedef double AT;
  for (int row = 0; row < n; ++row) {
    const Vec4d xv = X[row];
    AT acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    BLOCK_BRANCH
    for (int q = 0; q < 9; ++q) out[9 * row + q] = acc[q];
  }
}
extern "C" void batch_energy_terms(int n, const double* xs, const double* xts, const double* Pv, double* out) {
  std::vector<Vec4d> X = pack(n, xs), XT = pack(n, xts);
  struct { double pn0, pn1, pn2, po, dhat, kappa, fmu, feps, h2; } P{Pv[0], Pv[1], Pv[2], Pv[3], Pv[4], Pv[5],
                                                                   Pv[6], Pv[7], Pv[8]};
  struct { const Vec4d* xt; } in{XT.data()};
  for (int v = 0; v < n; ++v) {
    const Vec4d xv = X[v];
    double acc[2] = {0, 0};
    BATCH_ENERGY_BRANCH
    out[v] = acc[0];
  }
}
extern "C" void energy_terms(int n, const double* xs, const double* xts, const double* P, double* out) {
  SETUP
  for (int v = 0; v < n; ++v) {
    const Vec4d xv = X[v];
    double acc[2] = {0, 0};
    ENERGY_BRANCH
    out[v] = acc[0];
  }
}
'''


@pytest.fixture(scope="module")
def kernels(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    hdr = open(os.path.join(CSRC, "mls_internal.cuh")).read()
    a = hdr.index("// ---- lagged point-plane friction")
    helpers = hdr[a:hdr.index("}  // namespace mls", a)].replace("__device__ __forceinline__", "inline")
    asm = open(os.path.join(CSRC, "assemble.cu")).read()
    ele = open(os.path.join(CSRC, "elements.cu")).read()
    bat = open(os.path.join(CSRC, "batch.cu")).read()
    driver = (_DRIVER.replace("GRAD_BRANCH", _block(asm, "if constexpr (FRIC)", 0))
              .replace("BLOCK_BRANCH", _block(asm, "if constexpr (FRIC)", 1))
              .replace("BATCH_ENERGY_BRANCH", _block(bat, "if (P.fmu > 0.0)", 0))
              .replace("ENERGY_BRANCH", _block(ele, "if (in.fmu > 0.0)", 0)))
    d = tmp_path_factory.mktemp("friction_host")
    src, so = d / "friction_host.cpp", d / "friction_host.so"
    src.write_text(_PRELUDE + helpers + driver)
    res = subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(src)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    lib = C.CDLL(str(so))
    P = C.POINTER(C.c_double)

    def run(name, x, xt, params, width):
        out = np.zeros(len(x) * width)
        args = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, xt, params)]
        getattr(lib, name)(len(x), *[a.ctypes.data_as(P) for a in args], out.ctypes.data_as(P))
        return out.reshape(len(x), -1)
    return run


@pytest.mark.parametrize("plane", ["ground", "tilted"])
@pytest.mark.parametrize("slip", [0.0, 1e-7, 1e-5, 3e-5, 1e-3])
@pytest.mark.parametrize("bdf2", [False, True])
def test_kernel_friction_terms_match_oracle(kernels, plane, slip, bdf2):
    rng = np.random.default_rng(7 + int(1e7 * slip) + 2 * bdf2)
    dhat, kappa, mu, eps_v, h = 1e-3, 1e5, 0.45, 1e-3, 1.0 / 60
    h2 = (2 * h / 3) ** 2 if bdf2 else h * h          # the potentials' factor alpha h^2
    if plane == "ground":
        n, o, lo, tol = np.array([0.0, 0.0, 1.0]), 0.0, -2e-4, 1e-14
    else:
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        o, lo, tol = 0.1 * rng.normal(), 1e-4, 1e-11
    N = 60
    base = rng.normal(size=(N, 3))
    base -= (base @ n - o)[:, None] * n[None, :]
    xt = base + rng.uniform(lo, 2e-3, size=N)[:, None] * n[None, :]   # inside and beyond dhat
    x = xt + slip * rng.normal(size=(N, 3))
    x[::7] = xt[::7]                                                  # exactly no slip
    F = friction.GroundFriction(mu, eps_v, h, kappa, dhat, n, o, xt)
    assert np.any(F.lam > 0) and np.any(F.lam == 0)
    params = [n[0], n[1], n[2], o, dhat, kappa, mu, eps_v * h, h2]
    g = kernels("grad_terms", x, xt, params, 3)
    H = kernels("block_terms", x, xt, params, 9).reshape(N, 3, 3)
    E = kernels("energy_terms", x, xt, params, 1)[:, 0]
    E_batch = kernels("batch_energy_terms", x, xt, params, 1)[:, 0]
    g_o, H_o = F.gradient(x), h2 * F.hessian_blocks(x)
    assert np.abs(g - g_o).max() <= tol * np.abs(g_o).max()
    assert np.abs(H - H_o).max() <= tol * np.abs(H_o).max()
    assert E.sum() == pytest.approx(h2 * F.energy(x), rel=tol)
    assert E_batch.sum() == pytest.approx(h2 * F.energy(x), rel=tol)


_PREDICTOR_DRIVER = r'''
extern "C" void predictor_bdf2(int n, const double* x, const double* v, const double* xp, const double* vp,
                               const uint8_t* pinned, double h, double gx, double gy, double gz,
                               double* xt_out, double* xtil_out) {
  std::vector<Vec4d> xt(n), xtil(n), xk(n);
  auto body = [&](int i) PREDICTOR_BODY;
  for (int i = 0; i < n; ++i) body(i);
  for (int i = 0; i < n; ++i) {
    xt_out[3 * i] = xt[i].x; xt_out[3 * i + 1] = xt[i].y; xt_out[3 * i + 2] = xt[i].z;
    xtil_out[3 * i] = xtil[i].x; xtil_out[3 * i + 1] = xtil[i].y; xtil_out[3 * i + 2] = xtil[i].z;
    if (xk[i].x != xtil[i].x || xk[i].y != xtil[i].y || xk[i].z != xtil[i].z) xtil_out[3 * i] = NAN;
  }
}
'''


def test_kernel_bdf2_predictor_matches_oracle(tmp_path):
    """k_predictor_bdf2's body (one thread per vertex) against the oracle's
    BDF2 predictor (Sec. 3.1): x_tilde on free vertices, x^t on Dirichlet
    ones, and the Newton start equal to x_tilde."""
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    import synth
    from oracle import ip
    asm = open(os.path.join(CSRC, "assemble.cu")).read()
    body = _block(asm, "__global__ void k_predictor_bdf2(", 0)
    body = body.replace("const int i = blockIdx.x * blockDim.x + threadIdx.x;", "")
    src, so = tmp_path / "pred.cpp", tmp_path / "pred.so"
    src.write_text(_PRELUDE + _PREDICTOR_DRIVER.replace("PREDICTOR_BODY", body))
    res = subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(src)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    lib = C.CDLL(str(so))
    s = synth.tiny_scene(4, 3, 2, seed=11)                         # x = 0 face pinned
    rng = np.random.default_rng(12)
    x_prev = s.x0 + 1e-3 * rng.normal(size=s.x0.shape)
    v_prev = 0.3 * rng.normal(size=s.x0.shape)
    p = ip.Problem(s, integrator="bdf2", x_prev=x_prev, v_prev=v_prev)
    n = s.n_verts
    pinned = np.ascontiguousarray(s.dirichlet, dtype=np.uint8)
    assert pinned.any() and not pinned.all()
    xt, xtil = np.zeros((n, 3)), np.zeros((n, 3))
    P = C.POINTER(C.c_double)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (s.x0, s.v0, x_prev, v_prev)]
    g = [float(c) for c in s.gravity]
    lib.predictor_bdf2(C.c_int(n), *[a.ctypes.data_as(P) for a in arrs], pinned.ctypes.data_as(C.c_void_p),
                       C.c_double(s.dt), *[C.c_double(c) for c in g], xt.ctypes.data_as(P), xtil.ctypes.data_as(P))
    assert np.array_equal(xt, s.x0)
    assert np.allclose(xtil, p.x_tilde, rtol=0, atol=1e-15 * np.abs(p.x_tilde).max())
    assert np.array_equal(xtil[pinned.astype(bool)], s.x0[pinned.astype(bool)])
