"""The PCG loop's order-independent sums checked on the CPU by exact arithmetic.

Every dot product of the PCG loop (p.q, r.r, r.z) is accumulated on the GPU
as a fixed-point integer: each block partial x becomes round(x 2^(80-e))
(nearest, ties to even) in four 32-bit limbs added by atomics (``fix_add``),
and the consumer rebuilds the total rounded to the nearest double
(``fix_value``).  ``dbl_to_flt``, ``dbl_scale2`` and ``ratio`` convert and
divide on bit patterns.  All of this is integer code in mls_internal.cuh.

This test takes that section's source text unchanged, compiles it as host
C++ with g++ (the atomics become plain read-modify-writes, the bit casts
``memcpy``), and checks it against exact references that share nothing with
it: Python integers and ``fractions.Fraction`` for the rounded totals, and
numpy's float32 conversion (round to nearest even) for ``dbl_to_flt``.  The
claims checked are those the header states, with 2^e <= the scale estimate
< 2^(e+1): exact totals whatever the order of the partials, all 53 bits for
totals down to 2^(e-27), overflow flagged for partials from 2^(e+30) up,
non-finite partials flagged.  No GPU is used.
"""
import ctypes as C
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_13386_gb300", "csrc")

_PRELUDE = r'''
#include <cstdint>
#include <cstring>
#define __host__
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, sizeof v); return v; }
static inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, sizeof d); return d; }
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, sizeof f); return f; }
static inline int __clzll(long long v) { return v == 0 ? 64 : __builtin_clzll((unsigned long long)v); }
static inline unsigned long long __ldcg(const unsigned long long* p) { return *p; }
static inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  unsigned long long o = *p; *p = o + v; return o;
}
static inline unsigned long long atomicOr(unsigned long long* p, unsigned long long v) {
  unsigned long long o = *p; *p = o | v; return o;
}
'''

_DRIVER = r'''
extern "C" int host_fix_exponent(double x) { return fix_exponent(x); }
// adds xs[0..n) into one slot in the given order, then rebuilds the total
extern "C" double host_fix_sum(int n, const double* xs, const int* order, int e, int* bad) {
  unsigned long long slot[kFixSlotWords] = {0};
  for (int i = 0; i < n; ++i) fix_add(slot, xs[order[i]], e);
  const FixRaw r = fix_load(slot);
  bool b = false;
  const double v = fix_value(r, e, b);
  *bad = b ? 1 : 0;
  return v;
}
extern "C" void host_fix_words(int n, const double* xs, int e, unsigned long long* out) {
  unsigned long long slot[kFixSlotWords] = {0};
  for (int i = 0; i < n; ++i) fix_add(slot, xs[i], e);
  for (int k = 0; k < 5; ++k) out[k] = slot[k * kFixStride];
}
extern "C" float host_dbl_to_flt(double x) { return dbl_to_flt(x); }
extern "C" double host_dbl_scale2(double x, int d) { return dbl_scale2(x, d); }
extern "C" float host_ratio_f32(double a, double b) { return ratio<float>(a, b); }
'''


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    hdr = open(os.path.join(CSRC, "mls_internal.cuh")).read()
    a = hdr.index("// ---- order-independent sums for the PCG loop")
    body = hdr[a:hdr.index("// The state that opens PCG iteration", a)]
    d = tmp_path_factory.mktemp("fixed_point_host")
    src, so = d / "fixed_point_host.cpp", d / "fixed_point_host.so"
    src.write_text(_PRELUDE + body + _DRIVER)
    res = subprocess.run(["g++", "-O2", "-std=c++17", "-Wno-unknown-pragmas", "-shared", "-fPIC", "-o", str(so),
                          str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    lib = C.CDLL(str(so))
    lib.host_fix_exponent.restype = C.c_int
    lib.host_fix_exponent.argtypes = [C.c_double]
    lib.host_fix_sum.restype = C.c_double
    lib.host_fix_sum.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    lib.host_fix_words.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_ulonglong)]
    lib.host_dbl_to_flt.restype = C.c_float
    lib.host_dbl_to_flt.argtypes = [C.c_double]
    lib.host_dbl_scale2.restype = C.c_double
    lib.host_dbl_scale2.argtypes = [C.c_double, C.c_int]
    lib.host_ratio_f32.restype = C.c_float
    lib.host_ratio_f32.argtypes = [C.c_double, C.c_double]
    return lib


def _sum(lib, xs, e, order=None):
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    order = np.arange(len(xs), dtype=np.int32) if order is None else np.ascontiguousarray(order, dtype=np.int32)
    bad = C.c_int(0)
    v = lib.host_fix_sum(len(xs), xs.ctypes.data_as(C.POINTER(C.c_double)),
                         order.ctypes.data_as(C.POINTER(C.c_int)), e, C.byref(bad))
    return v, bad.value


def _exact(xs, e):
    """The definition: each partial rounded to the grid 2^(e-80) (nearest,
    ties to even), summed as integers, the total rounded to the nearest
    double (Python's int / int is correctly rounded)."""
    S = sum(round(Fraction(float(x)) * Fraction(2) ** (80 - e)) for x in xs)
    return S / 2 ** (80 - e) if 80 - e >= 0 else float(S * 2 ** (e - 80))


def test_fix_exponent_is_floor_log2(fx):
    rng = np.random.default_rng(5)
    for x in np.concatenate([10.0 ** rng.uniform(-300, 290, 200), [1.0, 2.0, 0.75, 2.0 ** 996]]):
        m, ex = math.frexp(x)  # x = m 2^ex, m in [0.5, 1)
        assert fx.host_fix_exponent(x) == ex - 1
    for x in [0.0, -1.0, float("inf"), float("nan"), 5e-324, 2.0 ** 997]:
        assert fx.host_fix_exponent(x) == 0


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1.0, 3.7e4, 1e40])
def test_fixed_point_total_is_exact_and_order_independent(fx, scale):
    """Mixed-sign partials spanning 2^-40 .. 2^29 of the estimate: the total
    equals the definition exactly, and every order gives the same bits."""
    rng = np.random.default_rng(int(scale * 1e3) % 2 ** 31 + 11)
    e = int(math.floor(math.log2(scale)))
    mags = scale * 2.0 ** rng.uniform(-40, 29, 3000)
    xs = mags * rng.choice([-1.0, 1.0], size=mags.size)
    ref = _exact(xs, e)
    v, bad = _sum(fx, xs, e)
    assert bad == 0
    assert v == ref
    for k in range(3):
        w, _ = _sum(fx, xs, e, rng.permutation(xs.size))
        assert np.float64(w).tobytes() == np.float64(v).tobytes()


def test_fixed_point_keeps_53_bits_down_to_2_pow_minus_27(fx):
    """A total as small as 2^-27 of the estimate, built from large partials
    that cancel, comes back as the exactly rounded double of the grid sum,
    i.e. with every bit of a double whose last place is on the grid."""
    rng = np.random.default_rng(9)
    e = 10
    for _ in range(50):
        target = 2.0 ** (e - 27) * (1 + rng.random())          # 53-bit value at 2^-27 of the scale
        target = float(np.round(target * 2.0 ** (80 - e)) / 2.0 ** (80 - e))
        big = 2.0 ** (e + 20) * rng.random(16)
        xs = np.concatenate([big, -big, [target]])
        v, bad = _sum(fx, xs, e, rng.permutation(xs.size))
        assert bad == 0 and v == target


def test_fixed_point_single_partials_round_trip(fx):
    """A single partial on the grid comes back unchanged; one below half a
    grid step vanishes; a tie rounds to even."""
    e = 0
    rng = np.random.default_rng(3)
    for x in 2.0 ** rng.uniform(-27, 29, 500) * rng.choice([-1, 1], 500):
        xq = float(np.round(x * 2.0 ** 80) / 2.0 ** 80)
        assert _sum(fx, [xq], e) == (xq, 0)
    assert _sum(fx, [2.0 ** -82], e) == (0.0, 0)                  # a quarter step
    assert _sum(fx, [2.0 ** -81], e) == (0.0, 0)                  # half a step: tie to even 0
    assert _sum(fx, [3 * 2.0 ** -81], e) == (2.0 ** -79, 0)       # 1.5 steps: tie to even 2


def test_fixed_point_flags_overflow_and_non_finite(fx):
    """Partials below 2^(e+30) fit (the largest double below it is 2^110 -
    2^57 grid steps); from 2^(e+30) up the slot's overflow word is set."""
    for e in (0, -40, 37):
        below = math.ldexp(1 - 2.0 ** -53, e + 30)
        v, bad = _sum(fx, [below, -below, math.ldexp(1.0, e)], e)
        assert bad == 0 and v == math.ldexp(1.0, e)
        assert _sum(fx, [math.ldexp(1.0, e + 30), 1.0], e)[1] == 1
    assert _sum(fx, [float("nan"), 1.0], e)[1] == 1
    assert _sum(fx, [float("inf")], e)[1] == 1


def test_fixed_point_limbs_of_a_negative_partial(fx):
    """-1 at e = 0 is -2^80: limb 2 holds -(2^16) as a 64-bit two's
    complement word, the others zero."""
    out = (C.c_ulonglong * 5)()
    xs = np.array([-1.0])
    fx.host_fix_words(1, xs.ctypes.data_as(C.POINTER(C.c_double)), 0, out)
    assert list(out) == [0, 0, (1 << 64) - (1 << 16), 0, 0]


def test_dbl_to_flt_rounds_to_nearest_even(fx):
    rng = np.random.default_rng(17)
    xs = np.concatenate([
        10.0 ** rng.uniform(-37, 38, 2000) * rng.choice([-1, 1], 2000),
        # exact ties between two floats: the 29 dropped bits are 1000...0
        [(1 + (2 * k + 1) * 2.0 ** -24) for k in range(8)],
        [1.0, -2.5, 3.4028234663852886e38, 1.1754943508222875e-38],
    ])
    for x in xs:
        assert np.float32(fx.host_dbl_to_flt(x)) == np.float32(x), x
    assert fx.host_dbl_to_flt(1e-39) == 0.0 and math.copysign(1, fx.host_dbl_to_flt(-1e-39)) < 0
    assert fx.host_dbl_to_flt(1e39) == float("inf") and fx.host_dbl_to_flt(-1e39) == -float("inf")
    assert fx.host_dbl_to_flt(3.4028235677973366e38) == float("inf")  # rounds past the largest float


def test_dbl_scale2_and_ratio(fx):
    rng = np.random.default_rng(23)
    for x, d in zip(10.0 ** rng.uniform(-200, 200, 300), rng.integers(-300, 300, 300)):
        assert fx.host_dbl_scale2(x, int(d)) == math.ldexp(x, int(d))
    assert fx.host_dbl_scale2(1.0, -1100) == 0.0 and fx.host_dbl_scale2(1.0, 1100) == float("inf")
    # ratio<float> of doubles far outside the float range, within 2 float ulps of the exact quotient
    for a, b in zip(10.0 ** rng.uniform(-300, 300, 300), 10.0 ** rng.uniform(-300, 300, 300)):
        q = Fraction(a) / Fraction(b)
        if not (2.0 ** -120 < q < 2.0 ** 120):
            continue
        r = fx.host_ratio_f32(a, b)
        assert abs(Fraction(float(r)) - q) <= 2 * 2.0 ** -23 * q
