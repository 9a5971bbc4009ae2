"""The mixed form's TF32 split (csrc/tf32_split.cuh), built for the host and checked on
the CPU against exact rational arithmetic.

The embedding kernels write every operand element x as TF32-exact big + small parts,
and the tensor-core GEMM sums big*big + big*small + small*big.  Bounds (u = 2^-11, the
TF32 rounding unit; FP32 rounds at 2^-24):

* tf32_round: the low 13 bits are zero and |tf32(x) - x| <= 2^-11 |x| (round to
  nearest, ties away from zero, at 10 stored mantissa bits);
* split of a float: x - big is exact in FP32, so |x - big - small| <= 2^-22 |x|;
* split of a double: one more FP32 rounding of x and of the remainder, so
  |x - big - small| <= 2^-22 (1 + 2^-10) |x|; the remainder x - big is formed as
  (f - big) + (x - f) from the float rounding f of x and its residual, which
  f32_round_with_residual takes from the bit pattern with integer operations:
  f must be the IEEE round-to-nearest-even float of x (numpy's cast) and the residual
  the float of the exact x - f;
* three-product sum: the dropped small*small term and the two split errors give
  |ab - (AB + A b_s + a_s B)| <= 3.1 * 2^-22 |ab|.  One TF32 product alone (the
  planted mistake) is off by about 2^-11 and fails it.
"""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

from helpers import build_host_probe

F = ctypes.POINTER(ctypes.c_float)
D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def probe():
    lib = build_host_probe("tf32_split_probe.cu", "tf32probe")
    lib.probe_tf32_round.argtypes = [F, F, ctypes.c_int]
    lib.probe_split_tf32f.argtypes = [F, F, F, ctypes.c_int]
    lib.probe_split_tf32.argtypes = [D, F, F, ctypes.c_int]
    lib.probe_f32_rn.argtypes = [D, F, ctypes.c_int]
    lib.probe_f32_residual.argtypes = [D, F, F, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    return lib


def model_tf32_round(x):
    """Round to nearest, ties away, at the 10-bit TF32 mantissa, on the FP32 bit pattern."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).copy()
    finite = (u & np.uint32(0x7f800000)) != np.uint32(0x7f800000)
    u[finite] = (u[finite] + np.uint32(0x1000)) & np.uint32(0xffffe000)
    return u.view(np.float32)


def values(rng, n, dtype):
    x = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n).astype(np.float64))
    return np.ascontiguousarray(x, dtype)


def run_round(probe, x):
    out = np.zeros_like(x)
    probe.probe_tf32_round(x.ctypes.data_as(F), out.ctypes.data_as(F), len(x))
    return out


def run_split(probe, x):
    big, small = np.zeros(len(x), np.float32), np.zeros(len(x), np.float32)
    if x.dtype == np.float32:
        probe.probe_split_tf32f(x.ctypes.data_as(F), big.ctypes.data_as(F), small.ctypes.data_as(F), len(x))
    else:
        probe.probe_split_tf32(x.ctypes.data_as(D), big.ctypes.data_as(F), small.ctypes.data_as(F), len(x))
    return big, small


def tf32_exact(v):
    return np.all((v.view(np.uint32) & np.uint32(0x1fff)) == 0)


def test_round_matches_model_and_bound(probe):
    rng = np.random.default_rng(11)
    x = values(rng, 20000, np.float32)
    # exact ties (low 13 bits 0x1000), their neighbours, zero, subnormals, infinities
    base = (x.view(np.uint32) & np.uint32(0xffffe000))
    ties = (base | np.uint32(0x1000)).view(np.float32)
    below = (base | np.uint32(0x0fff)).view(np.float32)
    special = np.array([0.0, -0.0, 1e-40, -1e-42, np.inf, -np.inf], np.float32)
    for v in (x, ties, below, special):
        got = run_round(probe, v)
        assert np.array_equal(got.view(np.uint32), model_tf32_round(v).view(np.uint32))
        assert tf32_exact(got[np.isfinite(got)])
    got = run_round(probe, x)
    for xi, gi in zip(x[:3000], got[:3000]):
        assert abs(Fraction(float(gi)) - Fraction(float(xi))) <= Fraction(1, 2 ** 11) * abs(Fraction(float(xi)))
    # ties go away from zero
    t = run_round(probe, ties)
    assert np.all(np.abs(t.astype(np.float64)) > np.abs(ties.astype(np.float64)))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_split_parts_exact_and_within_bound(probe, dtype):
    rng = np.random.default_rng(12)
    x = values(rng, 4000, dtype)
    big, small = run_split(probe, x)
    assert tf32_exact(big) and tf32_exact(small)
    bound = Fraction(1, 2 ** 22) * (1 if dtype == np.float32 else 1 + Fraction(1, 2 ** 10))
    for xi, bi, si in zip(x, big, small):
        X = Fraction(float(xi))
        assert abs(X - Fraction(float(bi)) - Fraction(float(si))) <= bound * abs(X)


def test_three_product_sum_within_bound(probe):
    rng = np.random.default_rng(13)
    a, b = values(rng, 3000, np.float64), values(rng, 3000, np.float64)
    ab_, as_ = run_split(probe, a)
    bb_, bs_ = run_split(probe, b)
    bound = Fraction(31, 10) / 2 ** 22
    worst_one_pass = Fraction(0)
    for i in range(len(a)):
        A, B = Fraction(float(a[i])), Fraction(float(b[i]))
        Ab, As, Bb, Bs = (Fraction(float(v)) for v in (ab_[i], as_[i], bb_[i], bs_[i]))
        assert abs(A * B - (Ab * Bb + Ab * Bs + As * Bb)) <= bound * abs(A * B)
        worst_one_pass = max(worst_one_pass, abs(A * B - Ab * Bb) / abs(A * B))
    assert worst_one_pass > bound * 100          # one TF32 pass would fail the bound


def edge_doubles(rng):
    """Doubles at the corners of the integer rounding: exact ties of the float rounding
    (dropped bits 2^28, kept bit even and odd), a carry out of the mantissa, the ends of
    the integer path's exponent range and just outside them, signs, zeros, subnormals
    and specials."""
    xs = []
    for E in (-74, -73, -20, 0, 1, 37, 126):
        for keep in (0, 1, 0x7FFFFE, 0x7FFFFF, 0x123456):
            for rem in (0, 1, 0x0FFFFFFF, 0x10000000, 0x10000001, 0x1FFFFFFF):
                bits = ((E + 1023) << 52) | (keep << 29) | rem
                x = np.array([bits], np.uint64).view(np.float64)[0]
                xs += [x, -x]
    for E in (-75, 127, 128, -1022, -1030):
        xs += [np.ldexp(1.5, E), -np.ldexp(1.25, E)]
    xs += [0.0, -0.0, 5e-324, -5e-324, np.inf, -np.inf, np.nan, 3.4e38, -3.5e38, 1e-300]
    xs += list(rng.standard_normal(2000) * np.exp2(rng.integers(-80, 130, 2000).astype(np.float64)))
    return np.ascontiguousarray(np.array(xs, np.float64))


def test_integer_float_rounding_equals_ieee(probe):
    x = edge_doubles(np.random.default_rng(14))
    got = np.zeros(len(x), np.float32)
    probe.probe_f32_rn(x.ctypes.data_as(D), got.ctypes.data_as(F), len(x))
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))


def test_integer_residual_is_the_float_of_the_exact_remainder(probe):
    x = edge_doubles(np.random.default_rng(15))
    n = len(x)
    f, r, ok = np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32)
    probe.probe_f32_residual(x.ctypes.data_as(D), f.ctypes.data_as(F), r.ctypes.data_as(F),
                             ok.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n)
    e = (x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7ff)
    assert np.array_equal(ok == 1, (e >= 949) & (e <= 1149))      # the documented range, exactly
    sel = ok == 1
    assert np.array_equal(f[sel].view(np.uint32), x[sel].astype(np.float32).view(np.uint32))
    exact_rem = x[sel] - f[sel].astype(np.float64)                  # exact in FP64
    assert np.array_equal(r[sel].view(np.uint32), exact_rem.astype(np.float32).view(np.uint32))


def test_split_of_edge_doubles_within_bound(probe):
    x = edge_doubles(np.random.default_rng(16))
    x = x[np.isfinite(x) & (np.abs(x) > 1e-30) & (np.abs(x) < 1e30)]
    big, small = run_split(probe, np.ascontiguousarray(x))
    assert tf32_exact(big) and tf32_exact(small)
    bound = Fraction(1, 2 ** 22) * (1 + Fraction(1, 2 ** 10))
    for xi, bi, si in zip(x, big, small):
        X = Fraction(float(xi))
        assert abs(X - Fraction(float(bi)) - Fraction(float(si))) <= bound * abs(X)
