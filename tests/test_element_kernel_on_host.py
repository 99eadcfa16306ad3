"""The element kernel's arithmetic checked on the CPU against the oracle.

``k_eval_elements`` (elements.cu) computes, per tet, the Neo-Hookean energy
vol psi(F), its gradient vol B^T vec(P) and the PSD-projected Hessian
vol B^T [dP/dF]_+ B (the material model of Sec. 4).  It projects dP/dF
analytically, in the frame of the SVD of F (two 3x3 Jacobi eigensolves per
tet).  The oracle instead eigen-decomposes the 9x9 dP/dF with a library
routine, so the two share no step.  ``k_expand_hessian`` spreads the kernel's
78-value layout back to 12x12.

This test takes the source text of both kernels and their helpers from
elements.cu unchanged, compiles it as host C++ with g++ (the CUDA qualifiers
defined away, the thread index supplied by a loop over the tets), and
compares per tet with ``oracle.elastic``.  The GPU parity tests check the same
kernel through the library; this one needs no GPU.

Tolerances: the host build agrees with the oracle to rounding (about 3e-15
of each tet's largest Hessian entry in float64, 1e-6 in float32), so this
test asks for 1e-13 on energies and 1e-12 on gradients and float64 Hessians,
and 1e-5 on float32 Hessians.  The GPU test allows more (1e-10, 2e-4) for the
device's fused multiply-adds and math library.  Two mistakes planted in the
oracle's results (the projection dropped, and mu and lambda swapped) are
checked to exceed these tolerances by far, so the comparison would see them.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import elastic

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_13386_gb300", "csrc")

_PRELUDE = r'''
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
using std::fabs;
using std::log;
using std::sqrt;
#define __host__
#define __device__
#define __global__
#define __forceinline__ inline
#define __launch_bounds__(...)
struct Vec4d { double x, y, z, w; };
struct Idx { int x; };
static Idx blockIdx, blockDim, threadIdx;
inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, sizeof d); return d; }
template <typename T, typename S> inline T load_as(S v) { return (T)v; }
'''

_DRIVER = r'''
template <typename CT>
static void eval_all(int t, const int* tets, const double* Dminv, const double* vol, const double* mu,
                     const double* lam, int n, const double* xs, double* energy, double* grad, double* H) {
  std::vector<Vec4d> X(n);
  for (int i = 0; i < n; ++i) X[i] = Vec4d{xs[3 * i], xs[3 * i + 1], xs[3 * i + 2], 0.0};
  std::vector<CT> h78((size_t)78 * t);
  ElemIn in{t, tets, Dminv, vol, mu, lam};
  blockIdx.x = 0;
  blockDim.x = 1;
  for (int e = 0; e < t; ++e) {
    threadIdx.x = e;
    k_eval_elements<CT, CT>(in, X.data(), energy, grad, h78.data());
  }
  for (int e = 0; e < t; ++e) {
    threadIdx.x = e;
    k_expand_hessian<CT>(t, h78.data(), H);
  }
}
extern "C" void eval_f64(int t, const int* tets, const double* Dminv, const double* vol, const double* mu,
                         const double* lam, int n, const double* xs, double* energy, double* grad, double* H) {
  eval_all<double>(t, tets, Dminv, vol, mu, lam, n, xs, energy, grad, H);
}
extern "C" void eval_f32(int t, const int* tets, const double* Dminv, const double* vol, const double* mu,
                         const double* lam, int n, const double* xs, double* energy, double* grad, double* H) {
  eval_all<float>(t, tets, Dminv, vol, mu, lam, n, xs, energy, grad, H);
}
'''


def _between(src, start, end):
    a = src.index(start)
    return src[a:src.index(end, a)]


def _hess_offset(hdr):
    """The header's constexpr hess_offset (78-value layout of the 4x4 vertex blocks)."""
    a = hdr.index("__host__ __device__ constexpr int hess_offset")
    return hdr[a:hdr.index("}", a) + 1] + "\n"


@pytest.fixture(scope="module")
def element_kernel(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    hdr = open(os.path.join(CSRC, "mls_internal.cuh")).read()
    ele = open(os.path.join(CSRC, "elements.cu")).read()
    body = _between(ele, "// ---- small dense helpers", "// ---- energy of the incremental potential")
    d = tmp_path_factory.mktemp("element_host")
    src, so = d / "element_host.cpp", d / "element_host.so"
    src.write_text(_PRELUDE + _hess_offset(hdr) + body + _DRIVER)
    res = subprocess.run(["g++", "-O2", "-std=c++17", "-Wno-unknown-pragmas", "-shared", "-fPIC", "-o", str(so),
                          str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    lib = C.CDLL(str(so))
    P = C.POINTER(C.c_double)
    Pi = C.POINTER(C.c_int)

    def run(precision, x, tets, vol, Dm_inv, mu, lam):
        t = len(tets)
        tets_soa = np.ascontiguousarray(np.asarray(tets, dtype=np.int32).T)          # [4][t]
        dm_soa = np.ascontiguousarray(np.asarray(Dm_inv).reshape(t, 9).T)             # [(3k+b)][t]
        E = np.zeros(t)
        g = np.zeros(12 * t)
        H = np.zeros((t, 12, 12))
        args = [np.ascontiguousarray(a, dtype=np.float64) for a in (dm_soa, vol, mu, lam, x)]
        getattr(lib, {"fp64": "eval_f64", "fp32": "eval_f32"}[precision])(
            t, tets_soa.ctypes.data_as(Pi), *[a.ctypes.data_as(P) for a in args[:4]], len(x),
            args[4].ctypes.data_as(P), E.ctypes.data_as(P), g.ctypes.data_as(P), H.ctypes.data_as(P))
        return E, g.reshape(12, t).T, H
    return run


def _case(compress, seed=31):
    s = synth.tiny_scene(4, 3, 2, seed=seed)
    rng = np.random.default_rng(seed)
    x = s.X + 0.002 * rng.normal(size=s.X.shape)
    if compress is not None:
        x = x * np.asarray(compress)[None, :]
    vol, Dm_inv = elastic.rest_shape(s.X, s.tets)
    mu, lam = elastic.lame(s.E, s.nu)
    return x, s.tets, vol, Dm_inv, mu, lam


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("compress", [None, (0.7, 1.0, 1.1), (1.3, 0.8, 0.9)])
def test_element_kernel_source_matches_oracle(element_kernel, precision, rtol, compress):
    x, tets, vol, Dm_inv, mu, lam = _case(compress)
    E, g, H = element_kernel(precision, x, tets, vol, Dm_inv, mu, lam)
    E_o = elastic.element_energy(x, tets, vol, Dm_inv, mu, lam)
    g_o = elastic.element_gradient(x, tets, vol, Dm_inv, mu, lam)
    H_o = elastic.element_hessian(x, tets, vol, Dm_inv, mu, lam, project=True)
    # energy and gradient are float64 in every precision mode
    assert np.allclose(E, E_o, rtol=1e-13, atol=1e-13 * np.abs(E_o).max())
    assert np.allclose(g, g_o, rtol=1e-12, atol=1e-12 * np.abs(g_o).max())
    scale = np.abs(H_o).max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(H - H_o) / scale) <= rtol
    assert np.allclose(H, np.swapaxes(H, 1, 2), atol=rtol * scale.max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_element_kernel_source_inverted_tets(element_kernel, precision):
    """Mirrored, every tet is inverted (J < 0): infinite energy, as in the
    oracle, and zero gradient and Hessian blocks."""
    x, tets, vol, Dm_inv, mu, lam = _case(None)
    x[:, 0] *= -1.0
    E, g, H = element_kernel(precision, x, tets, vol, Dm_inv, mu, lam)
    E_o = elastic.element_energy(x, tets, vol, Dm_inv, mu, lam)
    assert np.all(np.isposinf(E)) and np.all(np.isposinf(E_o))
    assert not np.any(g) and not np.any(H)


def test_planted_oracle_mistakes_exceed_the_tolerances(element_kernel):
    x, tets, vol, Dm_inv, mu, lam = _case((0.7, 1.0, 1.1))
    E, g, H = element_kernel("fp64", x, tets, vol, Dm_inv, mu, lam)
    H_o = elastic.element_hessian(x, tets, vol, Dm_inv, mu, lam, project=True)
    scale = np.abs(H_o).max(axis=(1, 2), keepdims=True)
    # projection dropped: the compressed block has indefinite tets
    H_raw = elastic.element_hessian(x, tets, vol, Dm_inv, mu, lam, project=False)
    assert np.max(np.abs(H - H_raw) / scale) > 1e3 * 1e-5
    # mu and lambda swapped
    E_sw = elastic.element_energy(x, tets, vol, Dm_inv, lam, mu)
    assert not np.allclose(E, E_sw, rtol=1e-10, atol=1e-10 * np.abs(E_sw).max())
    g_sw = elastic.element_gradient(x, tets, vol, Dm_inv, lam, mu)
    assert not np.allclose(g, g_sw, rtol=1e-10, atol=1e-10 * np.abs(g_sw).max())
