"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

FP64 form.  Tolerances: residuals agree to 1e-12 absolute (rounding of FP64
sums of at most ~1e5 terms of size <= 1e-2); energies to |dE| < 1e-8 Ha and
amplitudes to max|dt| < 1e-7 as the FP64 target states.
"""
import json
import os

import numpy as np
import pytest

import ccsd_synth as cs
from oracle import ccsd_k, driver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [
    cs.SynthSpec((1, 1, 1), 3, 5, 301, time_reversal=False, fock_offdiag=0.1),
    cs.SynthSpec((2, 1, 1), 2, 3, 302),
    cs.SynthSpec((3, 1, 1), 3, 5, 303, time_reversal=False, fock_offdiag=0.05),
    cs.SynthSpec((2, 2, 1), 2, 4, 304, time_reversal=False),
    cs.SynthSpec((2, 2, 2), 1, 2, 305, time_reversal=False, fock_offdiag=0.05),
    cs.SynthSpec((3, 2, 1), 5, 7, 306),
]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def solver(spec, inp, **cfg):
    from paper_1911_00242_gb300.binding import Solver
    arrays = {k: dev(v) for k, v in inp.items()}
    return Solver(spec.grid, spec.nocc, spec.nvir, arrays, **cfg), arrays


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: f"{s.grid}-o{s.nocc}-v{s.nvir}")
def test_residual_parity(lib, spec):
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    t1, t2 = cs.random_amplitudes(spec, 11)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    S, _ = solver(spec, inp)
    d1, d2 = dev(t1), dev(t2)
    r1 = torch.empty_like(d1)
    r2 = torch.empty_like(d2)
    S.residual(d1, d2, r1, r2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(r1.cpu().numpy(), R1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r2.cpu().numpy(), R2, rtol=0, atol=1e-12)
    assert S.launches() > 10


def test_first_update_is_mp2(lib):
    spec = cs.SynthSpec((3, 1, 1), 2, 4, 311)
    inp = cs.generate(spec)
    S, _ = solver(spec, inp)
    S.iterate(1)
    e = S.energy()
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    D1, D2 = driver.denominators(P)
    mp2 = 0.25 * np.sum(np.abs(inp["oovv"]) ** 2 / D2) / spec.nk
    assert abs(e - mp2) < 1e-13


@pytest.mark.parametrize("diis", [0, 6])
def test_chain_solve_parity(lib, diis):
    """The 1D chain workload (N_k=4, o=4, v=8) converged to 1e-8 on both sides."""
    spec = cs.spec_for("chain_k4_o4_v8")
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    ref = driver.solve(P, tol=1e-8, max_iter=100, diis_depth=diis)
    assert ref["converged"]
    S, _ = solver(spec, inp, diis_depth=diis, conv_tol=1e-8, max_iter=100)
    ok, iters, mr = S.solve()
    assert ok and mr < 1e-8
    assert iters == ref["iters"]
    e = S.energy()
    assert abs(e.real - ref["energies"][-1].real / spec.nk) < 1e-8
    t1 = torch.empty((spec.nk, spec.nocc, spec.nvir), dtype=torch.complex128, device="cuda")
    t2 = torch.empty((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, dtype=torch.complex128, device="cuda")
    S.get_amplitudes(t1, t2)
    assert abs(t1.cpu().numpy() - ref["t1"]).max() < 1e-7
    assert abs(t2.cpu().numpy() - ref["t2"]).max() < 1e-7
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "chain_k4_o4_v8.json")))
    assert abs(e.real - g["e_ccsd_per_cell"]) < 1e-8


def test_iterates_match_step_by_step(lib):
    spec = cs.SynthSpec((2, 2, 1), 3, 5, 321, time_reversal=False, fock_offdiag=0.05)
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    es = []
    driver.solve(P, n_iter=4, callback=lambda it, a, b, e: es.append(e / spec.nk))
    S, _ = solver(spec, inp)
    for n in range(4):
        S.iterate(1)
        e = S.energy()
        assert abs(e - es[n]) < 1e-12


def test_host_inputs_are_copied(lib):
    spec = cs.SynthSpec((2, 1, 1), 2, 3, 331)
    inp = cs.generate(spec)
    from paper_1911_00242_gb300.binding import Solver
    S = Solver(spec.grid, spec.nocc, spec.nvir, inp)          # numpy arrays: host memory
    S2, _ = solver(spec, inp)
    S.iterate(3)
    S2.iterate(3)
    assert S.energy() == S2.energy()


def test_invalid_arguments(lib):
    from paper_1911_00242_gb300.binding import CCSDError, Solver
    spec = cs.SynthSpec((2, 1, 1), 2, 3, 341)
    inp = cs.generate(spec)
    with pytest.raises(CCSDError):
        Solver((0, 1, 1), 2, 3, {k: dev(v) for k, v in inp.items()})
    with pytest.raises(CCSDError):
        Solver(spec.grid, 2, 3, {k: dev(v) for k, v in inp.items()}, diis_depth=1)
