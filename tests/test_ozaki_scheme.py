"""The Ozaki form's arithmetic, modelled exactly on the CPU (no GPU, no library).

The Ozaki form (`csrc/ozaki.cuh`) forms FP64-accurate products on the BF16 tensor
cores (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59 (2012) 95-118):

* every operand row gets a power-of-two scale 2^E > max|x| and is cut into s balanced
  base-128 digits (BF16 integers);
* the slice pairs (p, q) with p + q <= s - 1 are multiplied; every diagonal d = p + q
  has its own FP32 TMEM accumulator, which sums the products of all its pairs over a
  window of at most oz_kwin(s) K slices of 64 of one momentum chunk;
* each window is scaled by its power of two and added into a float pair (hi, lo) with
  TwoSum (Knuth); the FP64 epilogue multiplies hi + lo by the reference scales RA RB.

This module restates those steps in integer and rational arithmetic, with the
kernel's constants read from the headers, checks that the restated split equals the
kernels' own split code (csrc/ozaki_split.cuh, built for the host), and checks what
the form's accuracy rests on:

1. the digits are in range, are exact in BF16, and reconstruct x within 2^{E-7s-1};
2. every partial sum of a window is an integer of magnitude <= 2^24 (so the tensor
   core's FP32 accumulation is exact), and one more stage would break that;
3. the truncated pair sum is within the bound derived below of the exact product;
4. the schedule of units, K slices and windows forms every kept pair exactly once, and
   the split of a tile's units over CTAs is a partition;
5. the float-pair accumulation loses no more than its lo roundings.

Error bound (per product a b, row scales 2^Ea, 2^Eb).  With a^ the split value,
|a - a^| <= 2^{Ea-7s-1} and |a| < 2^Ea, so |ab - a^b^| <= 2^{Ea+Eb-7s}(1 + 2^{-7s-2}).
The dropped pairs have p + q = d >= s, hence p, q >= 1 and |v_p w_q| <= 2^12; there are
2s - 1 - d of them on diagonal d, each weighted 2^{-7(d+2)}.  Their sum is at most
2^{Ea+Eb-7s} c_s / 4 with c_s = sum_{j=0}^{s-2} (s-1-j) 2^{-7j}.  The bound per product
is therefore 2^{Ea+Eb-7s} (1 + 2^{-7s-2} + c_s / 4).
"""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from helpers import build_host_probe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_00242_gb300", "csrc")
HEADERS = [os.path.join(CSRC, "ozaki.cuh"), os.path.join(CSRC, "ozaki_split.cuh"),
           os.path.join(CSRC, "ozaki_schedule.cuh")]


def _kernel_constants():
    src = "".join(open(h).read() for h in HEADERS)

    def const(name):
        m = re.search(r"constexpr int %s = (-?\d+);" % name, src)
        assert m, name
        return int(m.group(1))

    return {
        "BK": const("OZ_BK"),
        "BITS": const("OZ_SLICE_BITS"),
        "MAX_SLICES": const("OZ_MAX_SLICES"),
        "EXP_MIN": const("OZ_EXP_MIN"),
        "EXP_MAX": const("OZ_EXP_MAX"),
        "MAX_SPLIT": const("OZ_MAX_SPLIT"),
    }


K = _kernel_constants()
BITS = K["BITS"]
BASE = 1 << BITS
HALF = BASE >> 1


def digit_bound(p):
    """Largest |v_p|: the top digit reaches 2^7, the balanced low digits 2^6."""
    return BASE if p == 0 else HALF


def diagonal_bound(s, d):
    """Largest |sum over the pairs of diagonal d of v_p w_q| for one K element."""
    return sum(digit_bound(p) * digit_bound(d - p) for p in range(d + 1) if p < s and d - p < s)


def oz_kwin(s):
    """The longest window (K slices of 64) whose partial sums stay within 2^24 on every
    kept diagonal, found by search from the digit bounds (not from the kernel's formula)."""
    w = 0
    while all((w + 1) * K["BK"] * diagonal_bound(s, d) <= 1 << 24 for d in range(s)) and w < 16:
        w += 1
    return w


# ---------------------------------------------------------------- the split
def row_exponent(values):
    """E with 2^E > max|x| (the exponent of the largest magnitude plus one), clamped."""
    m = float(np.max(np.abs(values))) if len(values) else 0.0
    if m == 0.0:
        return 0
    return max(K["EXP_MIN"], min(K["EXP_MAX"], int(np.frexp(m)[1])))


def split(x, s, E):
    """Balanced base-128 digits v_0 .. v_{s-1} of Y = rint(x 2^{7s-E}), least significant first."""
    Y = int(np.rint(np.ldexp(x, BITS * s - E)))
    v = [0] * s
    for p in range(s - 1, 0, -1):
        dg = ((Y + HALF) & (BASE - 1)) - HALF
        Y = (Y - dg) >> BITS
        v[p] = dg
    v[0] = Y
    return v


def split_value(v, E):
    return sum(Fraction(vp) * Fraction(2) ** (E - BITS * (p + 1)) for p, vp in enumerate(v))


def c_s(s):
    return sum(Fraction(s - 1 - j) / Fraction(BASE) ** j for j in range(s - 1))


def product_bound(Ea, Eb, s):
    return Fraction(2) ** (Ea + Eb - BITS * s) * (1 + Fraction(1, 2 ** (BITS * s + 2)) + c_s(s) / 4)


def rows(rng, n, k, lo_exp, hi_exp):
    """Rows whose magnitudes span 10^lo_exp .. 10^hi_exp, with a few exact powers of two."""
    x = rng.standard_normal((n, k)) * 10.0 ** rng.uniform(lo_exp, hi_exp, (n, 1))
    x[0, : k // 2] = np.ldexp(1.0, int(rng.integers(-40, 40)))
    return x


@pytest.mark.parametrize("s", [3, 5, 7, 8])
def test_split_digits_range_bf16_and_reconstruction(s):
    rng = np.random.default_rng(100 + s)
    X = rows(rng, 12, 40, -30, 30)
    for r in X:
        E = row_exponent(r)
        for x in r:
            v = split(x, s, E)
            assert all(-HALF <= d < HALF for d in v[1:])
            assert abs(v[0]) <= BASE
            # an integer of at most 8 significant bits: its FP32 pattern has a zero low half (BF16-exact)
            assert all(int(np.float32(d).view(np.uint32)) & 0xFFFF == 0 for d in v)
            assert abs(Fraction(x) - split_value(v, E)) <= Fraction(2) ** (E - BITS * s - 1)


def test_split_top_digit_reaches_its_bound():
    """|v_0| = 128 occurs (x just below 2^E), so the window bound must allow it."""
    for s in (3, 5, 7):
        E = 3
        x = np.nextafter(np.ldexp(1.0, E), 0.0)
        v = split(x, s, E)
        assert v[0] == BASE and all(d == 0 for d in v[1:])
        v = split(-x, s, E)
        assert v[0] == -BASE and all(d == 0 for d in v[1:])


def test_split_zero_and_clamped_rows():
    assert row_exponent(np.zeros(4)) == 0
    assert split(0.0, 7, 0) == [0] * 7
    assert row_exponent(np.array([1e-300])) == K["EXP_MIN"]
    assert row_exponent(np.array([1e300])) == K["EXP_MAX"]


# ---------------------------------------------------------------- the kernel's own split code
@pytest.fixture(scope="module")
def probe():
    """csrc/ozaki_split.cuh and csrc/ozaki_schedule.cuh built for the host (the same
    source the kernels use)."""
    lib = build_host_probe("oz_split_probe.cu", "ozprobe")
    dp = ctypes.POINTER(ctypes.c_double)
    lib.probe_row_exponent.argtypes = [dp, ctypes.c_int]
    lib.probe_row_exponent.restype = ctypes.c_int
    lib.probe_split.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint16)]
    lib.probe_scales.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_float)]
    lib.probe_kwin.argtypes = [ctypes.c_int]
    lib.probe_kwin.restype = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int)
    lib.probe_unit_range.argtypes = [ctypes.c_int] * 5 + [ip, ip]
    return lib


def kernel_split(probe, xs, s, E):
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    out = np.zeros(len(xs) * s, np.uint16)
    probe.probe_split(xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(xs), s, E,
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    digits = (out.astype(np.uint32) << 16).view(np.float32)
    assert np.all(digits == np.rint(digits))
    return digits.astype(np.int64).reshape(len(xs), s)


def kernel_row_exponent(probe, row):
    row = np.ascontiguousarray(row, dtype=np.float64)
    return probe.probe_row_exponent(row.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(row))


@pytest.mark.parametrize("s", [3, 5, 7, 8])
def test_kernel_split_code_equals_the_model(probe, s):
    """The embedding kernels' split (row exponent, fixed point, digits, BF16 patterns)
    gives the model's digits bit for bit, also at the top-digit bound, at exact ties of
    the rounding (to even), for zeros and for rows outside the exponent clamp."""
    rng = np.random.default_rng(500 + s)
    X = rows(rng, 10, 40, -30, 30)
    for r in X:
        E = row_exponent(r)
        assert kernel_row_exponent(probe, r) == E
        got = kernel_split(probe, r, s, E)
        assert [list(g) for g in got] == [split(x, s, E) for x in r]
    E = 3
    top = np.nextafter(np.ldexp(1.0, E), 0.0)
    k = np.arange(-40, 40, dtype=np.float64)
    ties = (k + 0.5) * np.ldexp(1.0, E - BITS * s)                # x 2^{7s-E} = k + 1/2 exactly
    special = np.concatenate([[0.0, -0.0, top, -top, np.ldexp(1.0, E - 1)], ties])
    got = kernel_split(probe, special, s, E)
    assert [list(g) for g in got] == [split(x, s, E) for x in special]
    for row in (np.array([0.0, 0.0]), np.array([1e-300, -2e-300]), np.array([3e300, 1.0]), np.array([5e-324])):
        assert kernel_row_exponent(probe, row) == row_exponent(row)


def test_kernel_scales_are_the_powers_of_two(probe):
    f, r = ctypes.c_double(0.0), ctypes.c_float(0.0)
    for s in (3, 7, 8):
        for E in (K["EXP_MIN"], -7, 0, 5, K["EXP_MAX"]):
            probe.probe_scales(s, E, ctypes.byref(f), ctypes.byref(r))
            assert f.value == 2.0 ** (BITS * s - E)
            assert r.value == 2.0 ** E


# ---------------------------------------------------------------- exact windows
@pytest.mark.parametrize("s", range(1, K["MAX_SLICES"] + 1))
def test_window_sizes_keep_fp32_exact_and_are_maximal(s):
    lim = 1 << 24
    w = oz_kwin(s)
    assert w >= 1
    assert all(w * K["BK"] * diagonal_bound(s, d) <= lim for d in range(s))
    # one more K slice breaks some diagonal, unless the 16-slice cap applies
    assert w == 16 or any((w + 1) * K["BK"] * diagonal_bound(s, d) > lim for d in range(s))


def test_diagonal_bounds_by_hand():
    """2^14 for diagonal 0; 2^12 (d + 3) for 1 <= d <= s - 1: pairs (0, d) and (d, 0) at
    2^13, the d - 1 others at 2^12."""
    for s in range(1, K["MAX_SLICES"] + 1):
        assert diagonal_bound(s, 0) == 1 << 14
        for d in range(1, s):
            assert diagonal_bound(s, d) == (d + 3) << 12
    assert [oz_kwin(s) for s in range(1, 9)] == [16, 16, 12, 10, 9, 8, 7, 6]


@pytest.mark.parametrize("s", [2, 3, 7, 8])
def test_worst_case_window_sums_exactly_in_fp32(s):
    """A full window of the largest digits on the diagonal with the largest bound: every
    FP32 prefix is exact, in pair-major (the MMA issue) and K-major order."""
    w = oz_kwin(s)
    d = max(range(s), key=lambda dd: diagonal_bound(s, dd))
    per_k = [digit_bound(p) * digit_bound(d - p) for p in range(d + 1)]
    n = w * K["BK"]
    for terms in (np.repeat(per_k, n), np.tile(per_k, n)):
        acc = np.float32(0.0)
        tot = 0
        for t in terms:
            acc = np.float32(acc + np.float32(t))
            tot += int(t)
            assert int(acc) == tot
        assert tot <= 1 << 24


def test_random_window_prefixes_exact_in_fp32():
    rng = np.random.default_rng(6)
    for s in (3, 7, 8):
        n = oz_kwin(s) * K["BK"]
        for d in (0, 1, s - 1):
            acc, tot = np.float32(0.0), 0
            for p in range(d + 1):
                a = rng.integers(-BASE, BASE + 1, n) if p == 0 else rng.integers(-HALF, HALF, n)
                bq = rng.integers(-BASE, BASE + 1, n) if d - p == 0 else rng.integers(-HALF, HALF, n)
                for t in a * bq:
                    acc = np.float32(acc + np.float32(t))
                    tot += int(t)
                    assert int(acc) == tot


# ---------------------------------------------------------------- truncated products
def pair_sum(va, vb, Ea, Eb, s, dmax):
    """2^{Ea+Eb} sum_{p+q<=dmax} v_p w_q 2^{-7(p+q+2)}, exactly."""
    tot = Fraction(0)
    for p in range(s):
        for q in range(s):
            if p + q <= dmax:
                tot += Fraction(va[p] * vb[q]) * Fraction(2) ** (Ea + Eb - BITS * (p + q + 2))
    return tot


@pytest.mark.parametrize("s", [3, 5, 7, 8])
def test_truncated_dot_within_bound(s):
    rng = np.random.default_rng(200 + s)
    A = rows(rng, 4, 48, -8, 8)
    B = rows(rng, 4, 48, -8, 8)
    for a in A:
        Ea = row_exponent(a)
        sa = [split(x, s, Ea) for x in a]
        for b in B:
            Eb = row_exponent(b)
            sb = [split(x, s, Eb) for x in b]
            exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
            got = sum(pair_sum(u, w, Ea, Eb, s, s - 1) for u, w in zip(sa, sb))
            assert abs(got - exact) <= len(a) * product_bound(Ea, Eb, s)


def test_dropping_the_last_kept_diagonal_breaks_the_bound():
    """The bound discriminates: forming only p + q <= s - 2 exceeds it.  Equal entries
    with large digits (v_0 = 100, v_p = 60) make every product's error the same sign."""
    s, E = 5, 2
    x = float(split_value([100] + [60] * (s - 1), E))
    a = np.full(48, x)
    Ea = row_exponent(a)
    assert Ea == E and split(x, s, E) == [100] + [60] * (s - 1)
    v = split(x, s, E)
    exact = len(a) * Fraction(x) ** 2
    bound = len(a) * product_bound(E, E, s)
    assert abs(len(a) * pair_sum(v, v, E, E, s, s - 1) - exact) <= bound
    assert abs(len(a) * pair_sum(v, v, E, E, s, s - 2) - exact) > bound


# ---------------------------------------------------------------- the kernel's schedule
def unit_range(nch, S, kstages, nsplit, split_idx):
    """The units [u0, u1) of one CTA: units are (chunk, window) in order, each window
    oz_kwin(S) K slices (the chunk's last one shorter); split by K-slice count."""
    W = oz_kwin(S)
    nw = -(-kstages // W)
    nunits = nch * nw
    if nsplit <= 1:
        return 0, nunits
    total = nch * kstages
    lo, hi = total * split_idx // nsplit, total * (split_idx + 1) // nsplit
    u0 = u1 = nunits
    for u in range(nunits):
        c, wi = divmod(u, nw)
        start = c * kstages + wi * W
        if start >= lo and u0 == nunits:
            u0 = u
        if start >= hi:
            u1 = u
            break
    return u0, max(u0, u1)


@pytest.mark.parametrize("nch,S,kstages", [(1, 7, 1), (1, 7, 4), (3, 7, 8), (2, 3, 2), (5, 8, 3), (1, 1, 1),
                                           (2, 7, 23)])
def test_unit_split_is_a_partition(nch, S, kstages):
    nunits = nch * -(-kstages // oz_kwin(S))
    for nsplit in range(1, K["MAX_SPLIT"] + 1):      # up to the most CTAs the kernel splits a tile over
        covered = []
        prev = 0
        for sp in range(nsplit):
            u0, u1 = unit_range(nch, S, kstages, nsplit, sp)
            assert u0 == prev and u0 <= u1 <= nunits
            covered.extend(range(u0, u1))
            prev = u1
        assert covered == list(range(nunits))


def test_kernel_schedule_code_equals_the_model(probe):
    """The GEMM kernel's window lengths and unit split (csrc/ozaki_schedule.cuh, built for
    the host) equal the model's, and the kernel's split is a partition by itself."""
    assert all(probe.probe_kwin(s) == oz_kwin(s) for s in range(1, K["MAX_SLICES"] + 1))
    u0, u1 = ctypes.c_int(0), ctypes.c_int(0)
    for nch, S, kst in [(1, 7, 1), (1, 7, 4), (3, 7, 8), (2, 3, 2), (5, 8, 3), (1, 1, 1), (27, 7, 6), (4, 7, 23)]:
        nunits = nch * -(-kst // oz_kwin(S))
        for nsplit in range(1, K["MAX_SPLIT"] + 1):      # up to the most CTAs the kernel splits a tile over
            prev = 0
            for sp in range(nsplit):
                probe.probe_unit_range(nch, S, kst, nsplit, sp, ctypes.byref(u0), ctypes.byref(u1))
                assert (u0.value, u1.value) == unit_range(nch, S, kst, nsplit, sp)
                assert u0.value == prev and u0.value <= u1.value <= nunits
                prev = u1.value
            assert prev == nunits


def schedule(nch, S, kstages):
    """The MMA issuer's windows: per (chunk, window), for each diagonal d, the list of
    (chunk, p, q, kst) products it sums, in issue order (K slice, then p)."""
    W = oz_kwin(S)
    wins = []
    for c in range(nch):
        for k0 in range(0, kstages, W):
            ks = range(k0, min(k0 + W, kstages))
            wins.append({d: [(c, p, d - p, k) for k in ks for p in range(d + 1)] for d in range(S)})
    return wins


@pytest.mark.parametrize("nch,S,kstages", [(1, 7, 40), (2, 7, 9), (3, 3, 17), (1, 8, 33)])
def test_schedule_forms_each_kept_pair_once(nch, S, kstages):
    wins = schedule(nch, S, kstages)
    seen = [st for w in wins for d in w for st in w[d]]
    want = [(c, p, q, k) for c in range(nch) for p in range(S) for q in range(S) if p + q <= S - 1
            for k in range(kstages)]
    assert sorted(seen) == sorted(want) and len(seen) == len(set(seen))
    for w in wins:
        for d, sts in w.items():
            ks = {st[3] for st in sts}
            assert 0 < len(ks) <= oz_kwin(S)
            assert all(st[0] == sts[0][0] and st[1] + st[2] == d for st in sts)


def model_gemm(Ach, Bch, s):
    """The kernel's arithmetic for one output element per (m, n): chunks of A' and B' rows
    (lists of 1-D arrays of length kstages * 64), exact windows, FP32 window factors
    relative to RA, RB, and the (hi, lo) TwoSum accumulation.  Returns, per (m, n),
    (hi, lo, RA, RB, exact sum of the scaled windows, sum of |lo| after each add)."""
    nch = len(Ach)
    kst = len(Ach[0][0]) // K["BK"]
    M, N = len(Ach[0]), len(Bch[0])
    Ea = [[row_exponent(Ach[c][m]) for m in range(M)] for c in range(nch)]
    Eb = [[row_exponent(Bch[c][n]) for n in range(N)] for c in range(nch)]
    V = [[np.array([[split(x, s, Ea[c][m])[p] for x in Ach[c][m]] for m in range(M)], dtype=np.int64)
          for p in range(s)] for c in range(nch)]
    W = [[np.array([[split(x, s, Eb[c][n])[q] for x in Bch[c][n]] for n in range(N)], dtype=np.int64)
          for q in range(s)] for c in range(nch)]
    out = {}
    for m in range(M):
        RA = max(2.0 ** Ea[c][m] for c in range(nch))
        for n in range(N):
            RB = max(2.0 ** Eb[c][n] for c in range(nch))
            hi, lo = np.float32(0.0), np.float32(0.0)
            xsum, lo_abs = Fraction(0), 0.0
            for wd in schedule(nch, s, kst):
                for d in range(s):
                    win = wd[d]             # the window's products of diagonal d
                    c = win[0][0]
                    acc = 0
                    for (_, p, q, k) in win:
                        sl = slice(k * K["BK"], (k + 1) * K["BK"])
                        part = V[c][p][m, sl] * W[c][q][n, sl]
                        acc_prefix = acc + np.cumsum(part)
                        assert np.max(np.abs(acc_prefix)) <= 1 << 24
                        acc = int(acc_prefix[-1])
                    v = np.float32(acc)
                    assert int(v) == acc
                    sa = np.float32(2.0 ** Ea[c][m] / RA)
                    sb = np.float32(2.0 ** Eb[c][n] / RB)
                    fa = np.float32(sa * np.float32(2.0 ** (-BITS * (d + 2))))
                    x = np.float32(np.float32(v * sb) * fa)
                    assert Fraction(float(x)) == Fraction(acc) * Fraction(float(sb)) * Fraction(float(fa))
                    xsum += Fraction(float(x))
                    t = np.float32(hi + x)
                    bp = np.float32(t - hi)
                    e = np.float32(np.float32(hi - np.float32(t - bp)) + np.float32(x - bp))
                    assert Fraction(float(t)) + Fraction(float(e)) == Fraction(float(hi)) + Fraction(float(x))
                    hi = t
                    lo = np.float32(lo + e)
                    lo_abs += abs(float(lo))
            out[m, n] = (hi, lo, RA, RB, xsum, lo_abs, Ea, Eb)
    return out


@pytest.mark.parametrize("s,nch,kst", [(7, 2, 2), (8, 1, 3), (5, 3, 1), (3, 1, 13), (7, 1, 9)])
def test_kernel_model_matches_exact_product(s, nch, kst):
    rng = np.random.default_rng(400 + s)
    Kc = kst * K["BK"]
    M = N = 3
    # chunks with different magnitudes, so RA / RB and the relative window factors matter
    Ach = [rng.standard_normal((M, Kc)) * 10.0 ** rng.uniform(-3, 3, (M, 1)) for _ in range(nch)]
    Bch = [rng.standard_normal((N, Kc)) * 10.0 ** rng.uniform(-3, 3, (N, 1)) for _ in range(nch)]
    out = model_gemm(Ach, Bch, s)
    for (m, n), (hi, lo, RA, RB, xsum, lo_abs, Ea, Eb) in out.items():
        exact = sum(Fraction(x) * Fraction(y) for c in range(nch) for x, y in zip(Ach[c][m], Bch[c][n]))
        scheme = xsum * Fraction(RA) * Fraction(RB)
        bound = sum(Kc * product_bound(Ea[c][m], Eb[c][n], s) for c in range(nch))
        assert abs(scheme - exact) <= bound
        # the float pair loses at most one FP32 rounding of lo per add
        got = (Fraction(float(hi)) + Fraction(float(lo))) * Fraction(RA) * Fraction(RB)
        assert abs(got - scheme) <= Fraction(lo_abs) * Fraction(2) ** -24 * (1 + Fraction(2) ** -23) \
            * Fraction(RA) * Fraction(RB)
        if s >= 7:
            # FP64-level: the GPU tests' tolerance, 1e-13 of sum |a||b|
            mag = sum(abs(Fraction(x) * Fraction(y)) for c in range(nch) for x, y in zip(Ach[c][m], Bch[c][n]))
            assert abs(got - exact) <= Fraction(1, 10 ** 13) * mag
