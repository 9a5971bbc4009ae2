"""Parity at the full size of the mixed-precision workload: 3x3x3 k grid
(N_k = 27), 8 occupied and 24 virtual spin orbitals per k, integrals stored
complex64 (vvvv 52 GB).  The full oracle cannot run at this size (its W~^abef
alone is 104 GB), so the residual (paper Sec. 2, Eqs. ori_EqSingle and
ori_EqDouble) is checked on sampled momentum blocks that the block oracle
computes one by one from the same inputs, in the launch configuration the
benchmark times (automatic work-memory layout: pooled tensor-core operands,
chunked ladder, W' slabs; the Ozaki form in the lean layout).  DIIS is off here
because it does not enter a residual evaluation.

Inputs are synthesized on the GPU by the input module (the generator's torch
evaluation, pinned to its numpy form on the CPU); amplitudes are random,
antisymmetric and k-conserving.  The FP64 and Ozaki forms solve the equations of
exactly the stored complex64 values (widened exactly), as the block oracle does.
Bars, relative to max|R| over the sampled blocks: mixed form 1e-5 (the small-grid
mixed bar), Ozaki form 1e-11 (its small-grid bar); FP64 form 1e-12 absolute (FP64
sums of at most ~1e5 terms, each side in its own order)."""
import pytest

import ccsd_synth as cs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R2_BLOCKS = [(0, 0, 0), (1, 5, 26), (13, 4, 13), (26, 26, 9)]
R1_KPOINTS = [0, 17]


@pytest.fixture(scope="module")
def grid333():
    """Inputs on the device, amplitudes, and the block oracle's R1 / R2 samples."""
    from oracle.ccsd_k_block import BlockProblem, BlockResidual
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if total < 250e9:
        pytest.skip("needs a GPU with about 280 GB")
    spec = cs.spec_for("grid333_o8_v24_c64")
    inp = cs.generate_torch(spec, "cuda")
    t1, t2 = cs.random_amplitudes_torch(spec, 77, "cuda")
    torch.cuda.empty_cache()
    host = {k: v.cpu().numpy() for k, v in inp.items()}
    B = BlockResidual(BlockProblem(spec.grid, spec.nocc, spec.nvir, host), t1.cpu().numpy(), t2.cpu().numpy())
    ref1 = {k: B.r1(k) for k in R1_KPOINTS}
    ref2 = {b: B.r2(*b) for b in R2_BLOCKS}
    del host, B
    scale = max(max(abs(x).max() for x in ref1.values()), max(abs(x).max() for x in ref2.values()))
    yield spec, inp, t1, t2, ref1, ref2, scale
    del inp, t1, t2
    torch.cuda.empty_cache()


def _residual(spec, inp, t1, t2, **cfg):
    from paper_1911_00242_gb300.binding import Solver
    S = Solver(spec.grid, spec.nocc, spec.nvir, inp, diis_depth=0, **cfg)
    r1, r2 = torch.empty_like(t1), torch.empty_like(t2)
    S.residual(t1, t2, r1, r2)
    torch.cuda.synchronize()
    got1 = {k: r1[k].cpu().numpy() for k in R1_KPOINTS}
    got2 = {b: r2[b].cpu().numpy() for b in R2_BLOCKS}
    S.close()
    del r1, r2
    torch.cuda.empty_cache()
    return got1, got2


def _errors(got1, got2, ref1, ref2):
    e1 = max(abs(got1[k] - ref1[k]).max() for k in R1_KPOINTS)
    e2 = max(abs(got2[b] - ref2[b]).max() for b in R2_BLOCKS)
    return e1, e2


def _antisym(got2):
    # blocks with ki = kj are antisymmetric in (i, j) within the block
    return max(abs(got2[b] + got2[b].transpose(1, 0, 2, 3)).max() for b in R2_BLOCKS if b[0] == b[1])


def test_grid333_mixed_residual_sampled(lib, grid333):
    from paper_1911_00242_gb300.binding import CCSD_MIXED
    spec, inp, t1, t2, ref1, ref2, scale = grid333
    got1, got2 = _residual(spec, inp, t1, t2, precision=CCSD_MIXED)
    e1, e2 = _errors(got1, got2, ref1, ref2)
    print(f"grid333 mixed residual: rel err R1 {e1 / scale:.2e}, R2 {e2 / scale:.2e} (of max|R| {scale:.3f})")
    assert e1 < 1e-5 * scale and e2 < 1e-5 * scale, (e1, e2, scale)
    assert _antisym(got2) < 1e-5 * scale


def test_grid333_ozaki_residual_sampled(lib, grid333):
    from paper_1911_00242_gb300.binding import CCSD_OZAKI
    spec, inp, t1, t2, ref1, ref2, scale = grid333
    # the lean layout (smaller operand pools) leaves room for the amplitude and residual
    # arrays beside the Ozaki handle
    got1, got2 = _residual(spec, inp, t1, t2, precision=CCSD_OZAKI, lean=1)
    e1, e2 = _errors(got1, got2, ref1, ref2)
    print(f"grid333 Ozaki residual: rel err R1 {e1 / scale:.2e}, R2 {e2 / scale:.2e}")
    assert e1 < 1e-11 * scale and e2 < 1e-11 * scale, (e1, e2, scale)
    assert _antisym(got2) < 1e-11 * scale


def test_grid333_fp64_residual_sampled(lib, grid333):
    spec, inp, t1, t2, ref1, ref2, scale = grid333
    got1, got2 = _residual(spec, inp, t1, t2)
    e1, e2 = _errors(got1, got2, ref1, ref2)
    print(f"grid333 FP64 residual: max|dR1| {e1:.1e}, max|dR2| {e2:.1e}")
    assert e1 < 1e-12 and e2 < 1e-12, (e1, e2)
    assert _antisym(got2) < 1e-12
