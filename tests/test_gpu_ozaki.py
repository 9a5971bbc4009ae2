"""GPU tests of the Ozaki form (CCSD_OZAKI): FP64-accurate contractions on the BF16
tensor cores.

* The GEMM alone (ccsd_oz_gemm) against numpy's complex128 product:
  - integer-valued operands whose slices and products are exact: the result must be
    bit-identical (this also checks that the tensor core's FP32 accumulation of the
    integer slice products is exact, which the scheme relies on);
  - random operands: the error obeys the scheme's bound, 4 (s + 2) 2^-7s K max|a| max|b|
    per output (slicing error of both operands plus the dropped slice pairs), and for
    s = 7 it is FP64-like (below 1e-13 of sum_k |a||b|);
  - rows of very different magnitude keep their own relative accuracy (row scales).
* Residuals against the oracle on small grids, default and lean layouts, complex128
  and complex64 integrals: within 1e-11 of max|R| (the FP64 form's 1e-12 absolute bar
  is met to within the scheme's truncation).
* A DIIS(6) solve of the chain workload: |dE| < 1e-8 Ha and max|dt| < 1e-7 against
  the oracle, the FP64 form's tolerances.
* The bounded-wait failure path of the Ozaki kernel.
"""
import numpy as np
import pytest

import ccsd_synth as cs
from oracle import ccsd_k, driver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def widened(inp):
    return {k: np.asarray(v, dtype=np.complex128) for k, v in inp.items()}


@pytest.mark.parametrize("M,Nc,K", [(128, 64, 256), (200, 130, 100), (1, 1, 1), (300, 257, 64)])
def test_oz_gemm_exact_on_integer_operands(lib, M, Nc, K):
    """Entries n 2^-12 with |n| < 2^15: three 7-bit slices hold them exactly under any row
    scale, and with s = 5 every slice pair is formed, so the product is exact."""
    from paper_1911_00242_gb300.binding import oz_gemm
    rng = np.random.default_rng(7 + M + K)
    def draw(r, c):
        re = rng.integers(-2 ** 15 + 1, 2 ** 15, size=(r, c))
        im = rng.integers(-2 ** 15 + 1, 2 ** 15, size=(r, c))
        return (re + 1j * im) * 2.0 ** -12
    A, B = draw(M, K), draw(Nc, K)
    C = oz_gemm(A, B, slices=5)
    ref = A @ B.T            # exact: integer multiples of 2^-24 below 2^53 units
    assert np.array_equal(C, ref)


def test_oz_gemm_exact_with_top_digits(lib):
    """Every entry (1 - 2^-20)(1 +- i) has the digits (128, 0, -2, 0, 0): top digits of
    the largest magnitude, and every dropped pair is zero, so the product is exact.  With
    5 slices a window is 9 K slices (64 real K each), so the 1024 real K span two."""
    from paper_1911_00242_gb300.binding import oz_gemm
    x = 1.0 - 2.0 ** -20
    A = np.full((128, 512), x + 1j * x)
    B = np.full((128, 512), x - 1j * x)
    C = oz_gemm(A, B, slices=5)
    assert np.array_equal(C, A @ B.T)
    assert C[0, 0] == 512 * 2 * x * x


def test_oz_gemm_exact_at_the_window_bound(lib):
    """The largest exact window: with 2 slices a window is 16 K slices, and the entries
    (1 - 2^-14)(1 +- i) (digits (128, -1)) make diagonal 0 of the real column sum 1024
    products of exactly 2^14 to 2^24, the largest integer range FP32 holds.  The result
    is the scheme's truncated product, exactly: per real K the kept pairs give
    128^2 2^-14 - 2 * 128 2^-21 = 1 - 2^-13 (the dropped pair (1, 1) is 2^-28)."""
    from paper_1911_00242_gb300.binding import oz_gemm
    x = 1.0 - 2.0 ** -14
    A = np.full((128, 512), x + 1j * x)
    B = np.full((64, 512), x - 1j * x)
    C = oz_gemm(A, B, slices=2)
    assert (C.real == 1024.0 - 0.125).all() and (C.imag == 0.0).all()


@pytest.mark.parametrize("slices", [3, 5, 7, 8])
@pytest.mark.parametrize("M,Nc,K", [(256, 256, 2048), (130, 70, 333)])
def test_oz_gemm_error_bound(lib, slices, M, Nc, K):
    from paper_1911_00242_gb300.binding import oz_gemm
    rng = np.random.default_rng(11 * slices + K)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((Nc, K)) + 1j * rng.standard_normal((Nc, K))
    C = oz_gemm(A, B, slices=slices)
    ref = A @ B.T
    amax = np.maximum(abs(A.real), abs(A.imag)).max(axis=1)
    bmax = np.maximum(abs(B.real), abs(B.imag)).max(axis=1)
    # each complex product is 4 real products (the real embedding); bound per real part
    bound = 4 * (slices + 2) * 2.0 ** (-7 * slices) * (2 * K) * np.outer(amax, bmax) * 4
    err = np.maximum(abs((C - ref).real), abs((C - ref).imag))
    assert (err <= bound + 1e-300).all(), (err / bound).max()
    if slices >= 7:
        absprod = abs(A) @ abs(B).T
        assert (abs(C - ref) <= 1e-13 * absprod).all()


def test_oz_gemm_row_scales(lib):
    """Rows spanning 1e-30 .. 1e10: each output keeps FP64-like accuracy relative to its
    own operand rows (per-row power-of-two scales)."""
    from paper_1911_00242_gb300.binding import oz_gemm
    rng = np.random.default_rng(3)
    M, Nc, K = 96, 80, 500
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((Nc, K)) + 1j * rng.standard_normal((Nc, K))
    A *= (10.0 ** rng.uniform(-15, 5, size=M))[:, None]
    B *= (10.0 ** rng.uniform(-15, 5, size=Nc))[:, None]
    A[5] = 0.0                                     # an all-zero row
    C = oz_gemm(A, B, slices=7)
    ref = A @ B.T
    absprod = abs(A) @ abs(B).T
    assert (abs(C - ref) <= 1e-13 * absprod + 1e-300).all()
    assert (C[5] == 0).all()


def test_oz_timeout_path(lib):
    """A stage that is never loaded: the bounded wait gives up, the kernel unwinds and
    the context stays usable."""
    from paper_1911_00242_gb300.binding import CCSD_ERR_TIMEOUT, oz_gemm
    assert lib.ccsd_oz_timeout_selftest() == CCSD_ERR_TIMEOUT
    A = np.ones((4, 8), dtype=np.complex128)
    assert np.array_equal(oz_gemm(A, A, slices=3), A @ A.T)


SPECS = [
    cs.SynthSpec((3, 1, 1), 3, 5, 601, time_reversal=False, fock_offdiag=0.05),
    cs.SynthSpec((3, 2, 1), 2, 4, 602),
    cs.SynthSpec((2, 2, 2), 2, 3, 603, time_reversal=False),
    cs.SynthSpec((2, 2, 1), 4, 12, 604),
    cs.SynthSpec((3, 1, 1), 2, 1, 605),
    cs.SynthSpec((2, 2, 1), 1, 2, 606),
]


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.grid}-o{s.nocc}-v{s.nvir}")
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ozaki_residual(lib, spec, dtype):
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_OZAKI, Solver
    inp = cs.generate(cs.SynthSpec(**{**spec.__dict__, "int_dtype": dtype}))
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, widened(inp))
    t1, t2 = cs.random_amplitudes(spec, 61)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    scale = max(abs(R1).max(), abs(R2).max())
    d1, d2 = dev(t1), dev(t2)
    for lean in (0, 1):
        S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_OZAKI,
                   lean=lean)
        r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        e1 = abs(r1.cpu().numpy() - R1).max() / scale
        e2 = abs(r2.cpu().numpy() - R2).max() / scale
        assert e1 < 1e-11 and e2 < 1e-11, (lean, e1, e2)
        # the native FP64 path of the same handle (W' slabs share the B pool when lean)
        S.set_precision(CCSD_FP64)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        assert abs(r1.cpu().numpy() - R1).max() < 1e-12 and abs(r2.cpu().numpy() - R2).max() < 1e-12
        S.set_precision(CCSD_OZAKI)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        assert abs(r2.cpu().numpy() - R2).max() / scale < 1e-11
        S.close()


def test_ozaki_slices_trade_accuracy(lib):
    """Fewer slices, larger error: s = 3 is near FP32-level, s = 8 FP64-level."""
    from paper_1911_00242_gb300.binding import CCSD_OZAKI, Solver
    spec = cs.SynthSpec((2, 2, 1), 4, 12, 607)
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    t1, t2 = cs.random_amplitudes(spec, 62)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    scale = max(abs(R1).max(), abs(R2).max())
    d1, d2 = dev(t1), dev(t2)
    errs = []
    for s in (3, 5, 8):
        S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_OZAKI,
                   oz_slices=s)
        r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        errs.append(abs(r2.cpu().numpy() - R2).max() / scale)
        S.close()
    assert errs[0] < 1e-5 and errs[1] < 1e-9 and errs[2] < 1e-12
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-14


def test_ozaki_solve_chain(lib):
    """Chain workload, DIIS(6): the Ozaki form converges to the oracle's fixed point within
    the FP64 form's tolerances (|dE| < 1e-8 Ha, max|dt| < 1e-7)."""
    from paper_1911_00242_gb300.binding import CCSD_OZAKI, Solver
    spec = cs.spec_for("chain_k4_o4_v8")
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    ref = driver.solve(P, tol=1e-8, max_iter=100, diis_depth=6)
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_OZAKI,
               diis_depth=6, conv_tol=1e-8, max_iter=100)
    ok, iters, mr = S.solve()
    assert ok and abs(iters - ref["iters"]) <= 1
    assert abs(S.energy().real - ref["energies"][-1].real / spec.nk) < 1e-8
    t1 = torch.empty((spec.nk, spec.nocc, spec.nvir), dtype=torch.complex128, device="cuda")
    t2 = torch.empty((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, dtype=torch.complex128, device="cuda")
    S.get_amplitudes(t1, t2)
    assert abs(t2.cpu().numpy() - ref["t2"]).max() < 1e-7


def test_ozaki_host_vvvv(lib):
    """vvvv in host memory, read in place by the FP64 W' kernel: the same residuals, bit
    for bit, as with vvvv on the device."""
    from paper_1911_00242_gb300.binding import CCSD_OZAKI, Solver
    for dtype in ("c128", "c64"):
        spec = cs.SynthSpec((3, 1, 1), 3, 5, 608, int_dtype=dtype)
        inp = cs.generate(spec)
        t1, t2 = cs.random_amplitudes(spec, 63)
        d1, d2 = dev(t1), dev(t2)
        for lean in (0, 1):
            out = []
            for on_host in (False, True):
                arrays = {k: dev(v) for k, v in inp.items()}
                if on_host:
                    arrays["vvvv"] = np.ascontiguousarray(inp["vvvv"])
                S = Solver(spec.grid, spec.nocc, spec.nvir, arrays, precision=CCSD_OZAKI, vvvv_on_host=on_host,
                           lean=lean)
                r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
                S.residual(d1, d2, r1, r2)
                torch.cuda.synchronize()
                out.append((r1.cpu().numpy(), r2.cpu().numpy()))
                S.close()
            assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("lean", [0, 1])
def test_mixed_with_ozaki_polish(lib, lean):
    """A mixed handle that carries the Ozaki steps: residuals of its three arithmetics on one
    handle (mixed, Ozaki, native FP64) against the oracle, then a DIIS(6) chain solve whose
    polish iterations run in the Ozaki form: |dE| < 1e-8 Ha and max|dt| < 1e-7 against the
    oracle's fixed point, the FP64 form's tolerances."""
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_MIXED, CCSD_OZAKI, Solver
    spec = cs.SynthSpec((2, 2, 1), 3, 6, 609, time_reversal=False)
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    t1, t2 = cs.random_amplitudes(spec, 64)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    scale = max(abs(R1).max(), abs(R2).max())
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_MIXED,
               polish_precision=CCSD_OZAKI, lean=lean)
    d1, d2 = dev(t1), dev(t2)
    r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
    for prec, tol in ((CCSD_MIXED, 1e-5), (CCSD_OZAKI, 1e-11), (CCSD_FP64, 1e-13), (CCSD_MIXED, 1e-5)):
        S.set_precision(prec)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        e = max(abs(r1.cpu().numpy() - R1).max(), abs(r2.cpu().numpy() - R2).max()) / scale
        assert e < tol, (prec, e)
    S.close()
    spec = cs.spec_for("chain_k4_o4_v8")
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    ref = driver.solve(P, tol=1e-10, max_iter=100, diis_depth=6)
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_MIXED,
               polish_precision=CCSD_OZAKI, diis_depth=6, conv_tol=1e-9, mixed_tol=1e-7, polish_iters=6,
               max_iter=100, lean=lean)
    ok, iters, mr = S.solve()
    assert ok and mr < 1e-9
    assert abs(S.energy().real - ref["energies"][-1].real / spec.nk) < 1e-8
    t1g = torch.empty((spec.nk, spec.nocc, spec.nvir), dtype=torch.complex128, device="cuda")
    t2g = torch.empty((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, dtype=torch.complex128, device="cuda")
    S.get_amplitudes(t1g, t2g)
    assert abs(t2g.cpu().numpy() - ref["t2"]).max() < 1e-7
