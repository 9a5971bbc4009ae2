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

The canonical blocks of the history (ki <= kj, ka <= kb) are checked on antisymmetric
amplitudes built here with this module's own momentum arithmetic: the weights count
every block once, the weighted inner product over canonical blocks equals the full
one, and unpacking through cmap (with its swaps and signs) gives back every block.
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
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.probe_canonical.argtypes = [ip, ip, ip, d, ip]
        _lib.probe_canonical.restype = ctypes.c_int
        _lib.probe_targets.argtypes = [ip, ip, ip]
        _lib.probe_targets.restype = ctypes.c_int
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


def canonical(grid):
    N = grid[0] * grid[1] * grid[2]
    dims = (ctypes.c_int * 3)(*grid)
    nc = ctypes.c_int(0)
    cblk = (ctypes.c_int * N ** 3)()
    cw = (ctypes.c_double * N ** 3)()
    cmap = (ctypes.c_int * N ** 3)()
    assert probe().probe_canonical(dims, ctypes.byref(nc), cblk, cw, cmap) == 1
    n = nc.value
    return np.array(cblk[:n]), np.array(cw[:n]), np.array(cmap[:])


def kb_table(grid):
    """kb = ki + kj - ka per block, from the grid coordinates (independent of the library)."""
    pts = [(a, b, c) for a in range(grid[0]) for b in range(grid[1]) for c in range(grid[2])]
    index = {p: k for k, p in enumerate(pts)}
    N = len(pts)
    kb = np.zeros((N, N, N), int)
    for ki, pi in enumerate(pts):
        for kj, pj in enumerate(pts):
            for ka, pa in enumerate(pts):
                kb[ki, kj, ka] = index[tuple((pi[d] + pj[d] - pa[d]) % grid[d] for d in range(3))]
    return kb


def antisymmetric_t2(rng, grid, o, v):
    """X - P(ij) X - P(ab) X + P(ij)P(ab) X for a random X: t2[ki,kj,ka](i,j,a,b)."""
    N = grid[0] * grid[1] * grid[2]
    kb = kb_table(grid)
    X = rng.standard_normal((N, N, N, o, o, v, v)) + 1j * rng.standard_normal((N, N, N, o, o, v, v))
    T = np.zeros_like(X)
    for ki in range(N):
        for kj in range(N):
            for ka in range(N):
                b = kb[ki, kj, ka]
                T[ki, kj, ka] = (X[ki, kj, ka] - X[kj, ki, ka].transpose(1, 0, 2, 3)
                                 - X[ki, kj, b].transpose(0, 1, 3, 2) + X[kj, ki, b].transpose(1, 0, 3, 2))
    return T


def test_canonical_blocks_weights_dot_and_unpack():
    rng = np.random.default_rng(9)
    for grid in [(1, 1, 1), (2, 1, 1), (3, 1, 1), (4, 1, 1), (2, 2, 1), (3, 2, 1), (2, 2, 2), (3, 3, 1)]:
        N = grid[0] * grid[1] * grid[2]
        o, v = 2, 3
        cblk, cw, cmap = canonical(grid)
        kb = kb_table(grid)
        assert cw.sum() == N ** 3
        for f in cblk:                                   # canonical: ki <= kj and ka <= kb
            ki, kj, ka = f // (N * N), (f // N) % N, f % N
            assert ki <= kj and ka <= kb[ki, kj, ka]
        T, U = antisymmetric_t2(rng, grid, o, v), antisymmetric_t2(rng, grid, o, v)
        Tf, Uf = T.reshape(N ** 3, o, o, v, v), U.reshape(N ** 3, o, o, v, v)
        full = np.real(np.vdot(T, U))
        canon = sum(w * np.real(np.vdot(Tf[f], Uf[f])) for f, w in zip(cblk, cw))
        assert abs(full - canon) <= 1e-12 * abs(full) + 1e-12
        if N > 1:                                        # unit weights (a plausible slip) miss it
            unweighted = sum(np.real(np.vdot(Tf[f], Uf[f])) for f in cblk)
            assert abs(full - unweighted) > 1e-6 * abs(full)
        for f in range(N ** 3):                          # unpack every block from its canonical one
            m = cmap[f]
            p, sij, sab = m >> 2, (m >> 1) & 1, m & 1
            blk = Tf[cblk[p]]
            if sij:
                blk = blk.transpose(1, 0, 2, 3)
            if sab:
                blk = blk.transpose(0, 1, 3, 2)
            sign = -1.0 if sij != sab else 1.0
            # the 4-term antisymmetrizer above rounds differently per block: 1e-13, not bits
            np.testing.assert_allclose(sign * blk, Tf[f], rtol=0, atol=1e-13)


def test_extrapolation_targets_write_every_block_once():
    """The device extrapolation writes each canonical element to the full blocks listed
    by diis_canonical_targets, with the swapped indices and the antisymmetry sign.  That
    scatter must write every full block exactly once and reproduce the antisymmetric t2,
    and list as many targets as the block's weight."""
    rng = np.random.default_rng(10)
    for grid in [(1, 1, 1), (2, 1, 1), (3, 1, 1), (4, 1, 1), (2, 2, 1), (3, 2, 1), (2, 2, 2), (3, 3, 1)]:
        N = grid[0] * grid[1] * grid[2]
        o, v = 2, 3
        cblk, cw, cmap = canonical(grid)
        dims = (ctypes.c_int * 3)(*grid)
        nc = ctypes.c_int(0)
        tg = (ctypes.c_int * (4 * N ** 3))()
        assert probe().probe_targets(dims, ctypes.byref(nc), tg) == 1
        assert nc.value == len(cblk)
        ctgt = np.array(tg[:4 * nc.value]).reshape(nc.value, 4)
        T = antisymmetric_t2(rng, grid, o, v)
        Tf = T.reshape(N ** 3, o, o, v, v)
        out = np.full_like(Tf, np.nan)
        writes = np.zeros(N ** 3, int)
        for p in range(nc.value):
            listed = [g for g in ctgt[p] if g >= 0]
            assert len(listed) == cw[p] and all(g >= 0 for g in ctgt[p][:len(listed)])
            src = Tf[cblk[p]]
            for g in listed:
                f, sij, sab = g >> 2, (g >> 1) & 1, g & 1
                blk = src
                if sij:
                    blk = blk.transpose(1, 0, 2, 3)
                if sab:
                    blk = blk.transpose(0, 1, 3, 2)
                out[f] = (-1.0 if sij != sab else 1.0) * blk
                writes[f] += 1
        assert np.all(writes == 1)
        np.testing.assert_allclose(out, Tf, rtol=0, atol=1e-13)
