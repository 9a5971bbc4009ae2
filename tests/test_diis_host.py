"""The library's DIIS coefficient solve (csrc/diis.h, host code), built for the host and
checked on the CPU.

Pulay extrapolation takes the coefficients c that minimise |sum_i c_i e_i| subject to
sum_i c_i = 1, from the Gram matrix B_ij = Re <e_i|e_j> of the last m update errors.
The checks do not restate the library's elimination:

* the bordered system [B -1; -1 0][c; l] = [0; -1] solved by LAPACK gives the same c;
* sum c = 1, and the combination is no longer than any single error vector nor than
  random affine combinations (the constrained minimum);
* a zero first error vector needs a row exchange and gives c = (1, 0);
* two identical error vectors make the system singular, which the solve reports.
"""
import ctypes

import numpy as np

from helpers import build_host_probe

_lib = None


def probe():
    global _lib
    if _lib is None:
        _lib = build_host_probe("diis_probe.cu", "diisprobe")
        d = ctypes.POINTER(ctypes.c_double)
        _lib.probe_diis.argtypes = [d, ctypes.c_int, d]
        _lib.probe_diis.restype = ctypes.c_int
    return _lib


def solve(B):
    B = np.ascontiguousarray(B, np.float64)
    m = B.shape[0]
    c = np.zeros(m)
    ok = probe().probe_diis(B.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m,
                            c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return bool(ok), c


def gram(E):
    return np.real(E.conj() @ E.T)


def test_coefficients_match_lapack_and_minimise():
    rng = np.random.default_rng(3)
    for m in range(2, 9):
        for trial in range(5):
            E = rng.standard_normal((m, 40)) + 1j * rng.standard_normal((m, 40))
            E *= np.exp2(rng.integers(-20, 20, (m, 1)))           # error vectors of very different size
            B = gram(E)
            ok, c = solve(B)
            assert ok
            K = np.zeros((m + 1, m + 1))
            K[:m, :m] = B
            K[:m, m] = K[m, :m] = -1.0
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            ref = np.linalg.solve(K, rhs)[:m]
            np.testing.assert_allclose(c, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
            assert abs(c.sum() - 1.0) < 1e-12
            r = np.linalg.norm(c @ E)
            assert r <= np.linalg.norm(E, axis=1).min() * (1 + 1e-12)
            for _ in range(20):
                w = rng.standard_normal(m)
                w /= w.sum()
                assert r <= np.linalg.norm(w @ E) * (1 + 1e-12)


def test_zero_leading_error_needs_a_row_exchange():
    E = np.zeros((2, 5))
    E[1] = [1.0, 2.0, 0.0, -1.0, 0.5]
    ok, c = solve(gram(E))
    assert ok and np.allclose(c, [1.0, 0.0], atol=1e-15)


def test_identical_errors_are_reported_singular():
    e = np.array([0.5, -1.0, 2.0, 0.25])
    ok, _ = solve(gram(np.stack([e, e, 2 * e])))
    assert not ok
