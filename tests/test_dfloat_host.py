"""The double-float arithmetic of the Ozaki form (csrc/dfloat.cuh), built for the host
and checked on the CPU against exact rational arithmetic.

The device build uses the FP32 intrinsics __fadd_rn, __fsub_rn, __fmul_rn and __fmaf_rn.
The host build of the same source uses plain FP32 operations and fmaf, compiled with
-ffp-contract=off, so each operation rounds once to nearest in both builds.  Checks:

* the results are normalized: |l| <= ulp(h) / 2;
* conversion from double keeps about 48 bits: |df(x) - x| <= 2^-47 |x|;
* the product and the fused multiply-add are within 2^-44 of the exact result
  (relative to |a b| and |a b| + |c|); the sum and difference are within 2^-44 of
  |a| + |b| (this sum adds the two low parts with one rounding, so under cancellation
  its bound is relative to the operands, not to the result);
* a planted mistake (the product without its low-part terms) fails the product bound.
"""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

from helpers import build_host_probe


@pytest.fixture(scope="module")
def probe():
    lib = build_host_probe("df_host_probe.cu", "dfprobe")
    f = ctypes.POINTER(ctypes.c_float)
    d = ctypes.POINTER(ctypes.c_double)
    for name in ("probe_df_add", "probe_df_sub", "probe_df_mul"):
        getattr(lib, name).argtypes = [f, f, f, ctypes.c_int]
    lib.probe_df_fma.argtypes = [f, f, f, f, ctypes.c_int]
    lib.probe_df_from_double.argtypes = [d, f, ctypes.c_int]
    return lib


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def random_df(rng, n, lo=-30, hi=30):
    """n double-floats (h, l) from doubles of random sign and exponent: h = fl32(x),
    l = fl32(x - h)."""
    x = rng.standard_normal(n) * np.exp2(rng.integers(lo, hi, n).astype(np.float64))
    h = x.astype(np.float32)
    l_ = (x - h.astype(np.float64)).astype(np.float32)
    return np.stack([h, l_], axis=1).reshape(-1).copy()


def value(p, i):
    return Fraction(float(p[2 * i])) + Fraction(float(p[2 * i + 1]))


def normalized(p, i):
    h, l_ = np.float32(p[2 * i]), np.float32(p[2 * i + 1])
    return abs(float(l_)) <= float(np.spacing(np.abs(h))) / 2


N = 4000
TOL = Fraction(1, 2 ** 44)


def test_add_sub_within_bound(probe):
    rng = np.random.default_rng(1)
    x, y = random_df(rng, N), random_df(rng, N, -20, 20)
    for fn, sign in ((probe.probe_df_add, 1), (probe.probe_df_sub, -1)):
        out = np.zeros(2 * N, np.float32)
        fn(_fp(x), _fp(y), _fp(out), N)
        for i in range(N):
            a, b = value(x, i), value(y, i)
            assert abs(value(out, i) - (a + sign * b)) <= TOL * (abs(a) + abs(b))
            assert normalized(out, i)


def test_cancellation_keeps_the_low_parts(probe):
    """a - a' for nearly equal a, a': the low parts carry the whole result."""
    rng = np.random.default_rng(2)
    x = random_df(rng, N)
    y = x.copy()
    y[1::2] = (y[1::2] * np.float32(0.5)).astype(np.float32)       # same h, half the l
    out = np.zeros(2 * N, np.float32)
    probe.probe_df_sub(_fp(x), _fp(y), _fp(out), N)
    for i in range(N):
        exact = value(x, i) - value(y, i)
        assert value(out, i) == exact


def test_mul_within_bound(probe):
    rng = np.random.default_rng(3)
    x, y = random_df(rng, N), random_df(rng, N)
    out = np.zeros(2 * N, np.float32)
    probe.probe_df_mul(_fp(x), _fp(y), _fp(out), N)
    for i in range(N):
        exact = value(x, i) * value(y, i)
        assert abs(value(out, i) - exact) <= TOL * abs(exact)
        assert normalized(out, i)


def test_fma_within_bound(probe):
    rng = np.random.default_rng(4)
    x, y, z = random_df(rng, N, -15, 15), random_df(rng, N, -15, 15), random_df(rng, N, -30, 30)
    out = np.zeros(2 * N, np.float32)
    probe.probe_df_fma(_fp(x), _fp(y), _fp(z), _fp(out), N)
    for i in range(N):
        ab, c = value(x, i) * value(y, i), value(z, i)
        assert abs(value(out, i) - (ab + c)) <= TOL * (abs(ab) + abs(c))
        assert normalized(out, i)


def test_conversion_from_double(probe):
    rng = np.random.default_rng(5)
    xs = rng.standard_normal(N) * np.exp2(rng.integers(-60, 60, N).astype(np.float64))
    out = np.zeros(2 * N, np.float32)
    probe.probe_df_from_double(xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _fp(out), N)
    for i in range(N):
        x = Fraction(float(xs[i]))
        assert abs(value(out, i) - x) <= Fraction(1, 2 ** 47) * abs(x)
        assert normalized(out, i)


def test_dropping_the_low_part_terms_breaks_the_product_bound(probe):
    """The bound discriminates: h_a h_b with its exact error, but without h_a l_b + l_a h_b,
    is off by about 2^-24 of the product."""
    rng = np.random.default_rng(6)
    x, y = random_df(rng, 200), random_df(rng, 200)
    bad = 0
    for i in range(200):
        ha, hb = Fraction(float(x[2 * i])), Fraction(float(y[2 * i]))
        exact = value(x, i) * value(y, i)
        if abs(ha * hb - exact) > TOL * abs(exact):
            bad += 1
    assert bad > 150
