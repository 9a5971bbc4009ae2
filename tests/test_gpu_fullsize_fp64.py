"""Parity at the full size of the FP64 workload: 2x2x2 k grid (N_k = 8), 8 occupied
and 32 virtual spin orbitals per k, complex128 integrals (vvvv 8.6 GB), DIIS(6) --
the configuration the benchmark times, with its launch plan (64 x 64 tiles over
M = N_k o^2 = 512 ladder rows, the antisymmetry-packed ladder in one W' slab, the
split-K choices at full K).

* Residual (paper Sec. 2, Eqs. ori_EqSingle and ori_EqDouble) at random
  antisymmetric, k-conserving amplitudes: R1 at every k and R2 on sampled momentum
  blocks, against the block oracle (form A, each block formed on its own).  Bars:
  FP64 form 1e-12 absolute elementwise (FP64 sums of at most ~1e5 terms of size
  <= 1e-2, summed in a different order on each side); Ozaki form 1e-11 of max|R|
  (its contractions are within ~2^-49 of sum |a||b|, its remaining GEMMs in
  double-float keep ~48 bits).
* Iterations (Sec. 4.4: the update t + R/D and the convergence quantity max|R|):
  the first two updates from t = 0 with DIIS(6) against values the oracle stored
  in tests/golden/grid222_o8_v32.json (written by tests/golden/make_golden.py).
  Bar: 1e-10 Ha on the energy per cell and 1e-10 relative on max|R|, well inside
  the FP64 target of 1e-8 Ha: after two updates the amplitudes carry only the
  residuals' rounding (1e-12 absolute above).
"""
import json
import os

import numpy as np
import pytest

import ccsd_synth as cs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAME = "grid222_o8_v32"
# (ki, kj, ka): kb = ki + kj - ka; (0,0,0) and (3,3,5) have ki = kj and ka = kb,
# (1,2,3) has kb = 0 != ka, (7,6,6) and (5,2,7) mix all four momenta
R2_BLOCKS = [(0, 0, 0), (1, 2, 3), (3, 3, 5), (7, 6, 6), (5, 2, 7), (6, 1, 4)]


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spec = cs.spec_for(NAME)
    inp = cs.generate(spec)
    dev = {k: torch.from_numpy(v).to("cuda") for k, v in inp.items()}
    return spec, inp, dev


@pytest.fixture(scope="module")
def reference(problem):
    from oracle.ccsd_k_block import BlockProblem, BlockResidual
    spec, inp, _ = problem
    t1, t2 = cs.random_amplitudes(spec, 41)
    B = BlockResidual(BlockProblem(spec.grid, spec.nocc, spec.nvir, inp), t1, t2)
    r1 = np.stack([B.r1(k) for k in range(spec.nk)])
    r2 = {b: B.r2(*b) for b in R2_BLOCKS}
    return t1, t2, r1, r2


def _residual(lib, problem, t1, t2, **cfg):
    from paper_1911_00242_gb300.binding import Solver
    spec, _, dev = problem
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, diis_depth=6, **cfg)
    d1 = torch.from_numpy(t1).to("cuda")
    d2 = torch.from_numpy(t2).to("cuda")
    r1, r2 = torch.empty_like(d1), torch.empty_like(d2)
    S.residual(d1, d2, r1, r2)
    torch.cuda.synchronize()
    out1 = r1.cpu().numpy()
    out2 = {b: r2[b].cpu().numpy() for b in R2_BLOCKS}
    # blocks with ki = kj are antisymmetric in (i, j) within the block
    anti = max(float(abs(out2[b] + out2[b].transpose(1, 0, 2, 3)).max()) for b in R2_BLOCKS if b[0] == b[1])
    S.close()
    return out1, out2, anti


def test_grid222_fp64_residual_sampled(lib, problem, reference):
    t1, t2, R1, R2 = reference
    r1, r2, anti = _residual(lib, problem, t1, t2)
    e1 = float(abs(r1 - R1).max())
    e2 = max(float(abs(r2[b] - R2[b]).max()) for b in R2_BLOCKS)
    print(f"grid222 FP64 residual: max|dR1| {e1:.1e}, max|dR2| {e2:.1e} on {len(R2_BLOCKS)} blocks")
    assert e1 < 1e-12 and e2 < 1e-12, (e1, e2)
    assert anti < 1e-12


def test_grid222_ozaki_residual_sampled(lib, problem, reference):
    from paper_1911_00242_gb300.binding import CCSD_OZAKI
    t1, t2, R1, R2 = reference
    r1, r2, anti = _residual(lib, problem, t1, t2, precision=CCSD_OZAKI)
    scale = max(float(abs(R1).max()), max(float(abs(x).max()) for x in R2.values()))
    e1 = float(abs(r1 - R1).max()) / scale
    e2 = max(float(abs(r2[b] - R2[b]).max()) for b in R2_BLOCKS) / scale
    print(f"grid222 Ozaki residual: rel err R1 {e1:.1e}, R2 {e2:.1e} (of max|R| {scale:.3f})")
    assert e1 < 1e-11 and e2 < 1e-11, (e1, e2)
    assert anti < 1e-11 * scale


@pytest.mark.parametrize("form", ["fp64", "ozaki"])
def test_grid222_first_updates_match_oracle(lib, problem, form):
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_OZAKI, Solver
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", NAME + ".json")))
    assert g["diis_depth"] == 6
    spec, _, dev = problem
    prec = CCSD_OZAKI if form == "ozaki" else CCSD_FP64
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, diis_depth=6, precision=prec)
    es, mrs = [], []
    for _ in range(2):
        done, mr = S.iterate(1)
        assert not done
        mrs.append(mr)
        es.append(S.energy())
    S.close()
    # the second call's max|R| is that of R(t0), the oracle's first recorded value
    for n in range(2):
        de = abs(es[n].real - g["e_per_cell_after_update"][n])
        print(f"{form} update {n + 1}: E {es[n].real:.12f}, |dE| {de:.1e}")
        assert de < 1e-10, (n, es[n], g["e_per_cell_after_update"][n])
        assert abs(es[n].imag - g["e_imag_per_cell_after_update"][n]) < 1e-10
    assert abs(mrs[1] - g["max_resid_after_update"][0]) < 1e-10 * g["max_resid_after_update"][0]
