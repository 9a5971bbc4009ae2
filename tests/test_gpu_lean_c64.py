"""GPU parity of the large-problem machinery at small sizes, against the oracle:

* the lean work-memory layout (ccsd_config.lean = 1): the FP64 ladder's W' in
  several momentum-pair slabs, the tensor-core operands in two shared pools
  rewritten every residual, the packed tensor-core ladder in several chunks;
* integral blocks stored complex64 (CCSD_C64): the FP64 form widens them
  exactly, so it must reproduce the oracle run on the widened values to FP64
  rounding; the mixed form reads them as stored.

Tolerances as in the FP64 and mixed parity tests: 1e-12 absolute for FP64
residuals, 1e-5 relative for mixed residuals, |dE| < 1e-6 Ha after polish."""
import numpy as np
import pytest

import ccsd_synth as cs
from oracle import ccsd_k, driver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [
    cs.SynthSpec((3, 1, 1), 3, 5, 501, time_reversal=False, fock_offdiag=0.05),
    cs.SynthSpec((3, 2, 1), 2, 4, 502),
    cs.SynthSpec((2, 2, 2), 2, 3, 503, time_reversal=False),
]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def widened(inp):
    return {k: np.asarray(v, dtype=np.complex128) for k, v in inp.items()}


def residual_pair(spec, inp, seed, **cfg):
    from paper_1911_00242_gb300.binding import Solver
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, widened(inp))
    t1, t2 = cs.random_amplitudes(spec, seed)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, **cfg)
    d1, d2 = dev(t1), dev(t2)
    r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
    S.residual(d1, d2, r1, r2)
    torch.cuda.synchronize()
    return S, (d1, d2, r1, r2), R1, R2


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.grid}-o{s.nocc}-v{s.nvir}")
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_lean_and_c64_fp64_residual(lib, spec, dtype):
    inp = cs.generate(cs.SynthSpec(**{**spec.__dict__, "int_dtype": dtype}))
    for lean in (0, 1):
        S, (d1, d2, r1, r2), R1, R2 = residual_pair(spec, inp, 51, lean=lean)
        np.testing.assert_allclose(r1.cpu().numpy(), R1, rtol=0, atol=1e-12)
        np.testing.assert_allclose(r2.cpu().numpy(), R2, rtol=0, atol=1e-12)


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.grid}-o{s.nocc}-v{s.nvir}")
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_lean_and_c64_mixed_residual(lib, spec, dtype):
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_MIXED
    inp = cs.generate(cs.SynthSpec(**{**spec.__dict__, "int_dtype": dtype}))
    for lean in (0, 1):
        S, (d1, d2, r1, r2), R1, R2 = residual_pair(spec, inp, 52, precision=CCSD_MIXED, lean=lean)
        scale = max(abs(R1).max(), abs(R2).max())
        e1 = abs(r1.cpu().numpy() - R1).max() / scale
        e2 = abs(r2.cpu().numpy() - R2).max() / scale
        assert e1 < 1e-5 and e2 < 1e-5, (lean, e1, e2)
        # the same handle in FP64 (the polish path: W' slabs in the shared pool when lean)
        S.set_precision(CCSD_FP64)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        assert abs(r2.cpu().numpy() - R2).max() < 1e-12
        assert abs(r1.cpu().numpy() - R1).max() < 1e-12
        # and back: the pooled operands are rebuilt from scratch every residual
        S.set_precision(CCSD_MIXED)
        S.residual(d1, d2, r1, r2)
        torch.cuda.synchronize()
        assert abs(r2.cpu().numpy() - R2).max() / scale < 1e-5


def test_lean_c64_mixed_solve_chain(lib):
    """Chain workload with complex64 integrals in the lean layout: mixed iterations,
    DIIS(6) on canonical blocks, two FP64 polish iterations; |dE| < 1e-6 Ha against
    the oracle on the widened integrals."""
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Solver
    spec = cs.SynthSpec(**{**cs.spec_for("chain_k4_o4_v8").__dict__, "int_dtype": "c64"})
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, widened(inp))
    ref = driver.solve(P, tol=1e-10, max_iter=100, diis_depth=6)
    e_ref = ref["energies"][-1].real / spec.nk
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_MIXED,
               diis_depth=6, conv_tol=1e-9, mixed_tol=1e-7, polish_iters=2, max_iter=100, lean=1)
    ok, iters, mr = S.solve()
    assert ok
    assert abs(S.energy().real - e_ref) < 1e-6


def test_c64_fp64_solve_chain(lib):
    """FP64 form on complex64-stored integrals converges to the oracle's fixed point of
    the widened integrals: |dE| < 1e-8 Ha, max|dt| < 1e-7, same iteration count."""
    from paper_1911_00242_gb300.binding import Solver
    spec = cs.SynthSpec(**{**cs.spec_for("chain_k4_o4_v8").__dict__, "int_dtype": "c64"})
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, widened(inp))
    ref = driver.solve(P, tol=1e-8, max_iter=100, diis_depth=6)
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, diis_depth=6,
               conv_tol=1e-8, max_iter=100, lean=1)
    ok, iters, mr = S.solve()
    assert ok and iters == ref["iters"]
    assert abs(S.energy().real - ref["energies"][-1].real / spec.nk) < 1e-8
    t1 = torch.empty((spec.nk, spec.nocc, spec.nvir), dtype=torch.complex128, device="cuda")
    t2 = torch.empty((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, dtype=torch.complex128, device="cuda")
    S.get_amplitudes(t1, t2)
    assert abs(t2.cpu().numpy() - ref["t2"]).max() < 1e-7


@pytest.mark.parametrize("spec", [cs.SynthSpec((3, 1, 1), 2, 1, 511), cs.SynthSpec((2, 2, 1), 1, 2, 512),
                                  cs.SynthSpec((1, 1, 1), 1, 1, 513, time_reversal=False)],
                         ids=["v1", "o1", "o1v1"])
def test_degenerate_sizes_both_forms(lib, spec):
    """One virtual or one occupied spin orbital per k: the packed (e < f, a < b, m < n)
    index lists are empty, so only the momentum-pair halves of the contractions remain."""
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_MIXED
    inp = cs.generate(spec)
    S, (d1, d2, r1, r2), R1, R2 = residual_pair(spec, inp, 53)
    assert abs(r1.cpu().numpy() - R1).max() < 1e-12 and abs(r2.cpu().numpy() - R2).max() < 1e-12
    for lean in (0, 1):
        S, (d1, d2, r1, r2), R1, R2 = residual_pair(spec, inp, 53, precision=CCSD_MIXED, lean=lean)
        scale = max(abs(R1).max(), abs(R2).max(), 1e-30)
        assert abs(r1.cpu().numpy() - R1).max() / scale < 1e-5
        assert abs(r2.cpu().numpy() - R2).max() / scale < 1e-5


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_vvvv_read_in_place_from_host(lib, dtype):
    """vvvv_on_host: the kernels read a host vvvv in place (mapped pinned memory): the
    same residuals, bit for bit, as with vvvv in device memory, in both forms and (lean)
    with the ladder split into several chunks."""
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Solver
    spec = cs.SynthSpec((3, 1, 1), 3, 5, 521, int_dtype=dtype)
    inp = cs.generate(spec)
    t1, t2 = cs.random_amplitudes(spec, 54)
    d1, d2 = dev(t1), dev(t2)
    for prec, lean in ((0, 0), (CCSD_MIXED, 0), (CCSD_MIXED, 1)):
        out = []
        for on_host in (False, True):
            arrays = {k: dev(v) for k, v in inp.items()}
            if on_host:
                arrays["vvvv"] = np.ascontiguousarray(inp["vvvv"])        # pageable host memory
            S = Solver(spec.grid, spec.nocc, spec.nvir, arrays, precision=prec, vvvv_on_host=on_host, lean=lean)
            r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
            S.residual(d1, d2, r1, r2)
            torch.cuda.synchronize()
            out.append((r1.cpu().numpy(), r2.cpu().numpy()))
            S.close()
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
