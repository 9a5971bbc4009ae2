"""Mixed form: tcgen05 TF32 tensor-core contractions (ladder, ring) and FP32
CUDA-core contractions, FP64 update/DIIS/energy, FP64 polish.

Tolerances: the split-TF32 GEMM keeps ~21 mantissa bits, so a residual of
size |R| carries errors of about 1e-6 |R|; the polished energy must agree
with the FP64 oracle to |dE| < 1e-6 Ha (the mixed-form target)."""
import ctypes

import numpy as np
import pytest

import ccsd_synth as cs
from oracle import ccsd_k, driver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# split TF32 is limited by FP32 accumulation (~eps_32 sqrt(2K) relative), plain TF32 by its
# 10-bit mantissa
@pytest.mark.parametrize("M,N,K,terms,tol", [(128, 128, 16, 3, 2e-5), (128, 128, 16, 1, 2e-3),
                                             (200, 300, 100, 3, 2e-5), (64, 1024, 1024, 3, 3e-5),
                                             (333, 129, 37, 1, 2e-3)])
def test_tensor_core_gemm_selftest(lib, M, N, K, terms, tol):
    err = ctypes.c_double(-1.0)
    rc = lib.ccsd_tc_selftest(M, N, K, terms, 7, ctypes.byref(err))
    assert rc == 0, rc
    assert 0 <= err.value < tol, err.value


MIXED = [
    cs.SynthSpec((2, 1, 1), 2, 3, 402),
    cs.SynthSpec((2, 2, 1), 3, 5, 404, time_reversal=False, fock_offdiag=0.05),
    cs.SynthSpec((3, 1, 1), 4, 8, 403),
    cs.SynthSpec((2, 2, 2), 2, 4, 405, time_reversal=False),
]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("spec", MIXED, ids=lambda s: f"{s.grid}-o{s.nocc}-v{s.nvir}")
def test_mixed_residual_parity(lib, spec):
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Solver
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    t1, t2 = cs.random_amplitudes(spec, 12)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_MIXED)
    d1, d2 = dev(t1), dev(t2)
    r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
    S.residual(d1, d2, r1, r2)
    torch.cuda.synchronize()
    scale = max(abs(R1).max(), abs(R2).max())
    e1 = abs(r1.cpu().numpy() - R1).max() / scale
    e2 = abs(r2.cpu().numpy() - R2).max() / scale
    assert e1 < 1e-5 and e2 < 1e-5, (e1, e2)
    # the same handle in FP64 reproduces the oracle to rounding
    S.set_precision(0)
    S.residual(d1, d2, r1, r2)
    torch.cuda.synchronize()
    assert abs(r2.cpu().numpy() - R2).max() < 1e-12


def test_mixed_solve_chain_energy(lib):
    """Chain workload: mixed iterations to 1e-7, two FP64 polish iterations, |dE| < 1e-6 Ha."""
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Solver
    spec = cs.spec_for("chain_k4_o4_v8")
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    ref = driver.solve(P, tol=1e-10, max_iter=100, diis_depth=6)
    e_ref = ref["energies"][-1].real / spec.nk
    S = Solver(spec.grid, spec.nocc, spec.nvir, {k: dev(v) for k, v in inp.items()}, precision=CCSD_MIXED,
               diis_depth=6, conv_tol=1e-9, mixed_tol=1e-7, polish_iters=2, max_iter=100)
    ok, iters, mr = S.solve()
    assert ok
    e = S.energy()
    assert abs(e.real - e_ref) < 1e-6, (e.real, e_ref)
