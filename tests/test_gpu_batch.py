"""Batched form: independent problems of uneven size in grouped persistent launches.

Each member must give the result it gives alone: FP64 energies to 1e-12 (the
grouped kernel runs the same tile arithmetic; only split-K partial sums may be
ordered differently), mixed energies to 1e-6 of the FP64 oracle."""
import numpy as np
import pytest

import ccsd_synth as cs
from oracle import ccsd_k, driver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [
    cs.SynthSpec((1, 1, 1), 4, 8, 2001),
    cs.SynthSpec((2, 1, 1), 3, 5, 2002),
    cs.SynthSpec((2, 2, 1), 2, 4, 2003, time_reversal=False),
    cs.SynthSpec((4, 1, 1), 4, 6, 2004),
    cs.SynthSpec((1, 1, 1), 2, 3, 2005),
    cs.SynthSpec((2, 1, 1), 5, 9, 2006),
]


def dev(inp):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to("cuda") for k, v in inp.items()}


def test_batch_members_match_standalone(lib):
    from paper_1911_00242_gb300.binding import BatchSolver, Solver
    inps = [cs.generate(s) for s in SPECS]
    devs = [dev(i) for i in inps]
    B = BatchSolver([(s.grid, s.nocc, s.nvir, d) for s, d in zip(SPECS, devs)], conv_tol=1e-30)
    B.iterate(4)
    eb = B.energies()
    for s, d, e in zip(SPECS, devs, eb):
        S = Solver(s.grid, s.nocc, s.nvir, d, conv_tol=1e-30)
        S.iterate(4)
        assert abs(S.energy() - e) < 1e-12, (s, S.energy(), e)
        S.close()
    n_launch, cfgs = B.stats()
    assert n_launch > 0
    B.close()


def test_batch_converges_each_member_to_oracle(lib):
    from paper_1911_00242_gb300.binding import BatchSolver
    specs = SPECS[:4]
    inps = [cs.generate(s) for s in specs]
    B = BatchSolver([(s.grid, s.nocc, s.nvir, dev(i)) for s, i in zip(specs, inps)], conv_tol=1e-9)
    done, mr = B.iterate(200)
    assert all(done), (done, mr)
    eb = B.energies()
    for s, inp, e in zip(specs, inps, eb):
        P = ccsd_k.Problem(s.grid, s.nocc, s.nvir, inp)
        ref = driver.solve(P, tol=1e-9, max_iter=200)
        assert abs(e.real - ref["energies"][-1].real / s.nk) < 1e-8
    B.close()


def test_mixed_batch_energy(lib):
    from paper_1911_00242_gb300.binding import CCSD_MIXED, BatchSolver
    specs = [SPECS[1], SPECS[3], SPECS[5]]
    inps = [cs.generate(s) for s in specs]
    B = BatchSolver([(s.grid, s.nocc, s.nvir, dev(i)) for s, i in zip(specs, inps)], conv_tol=1e-7,
                    precision=CCSD_MIXED)
    done, mr = B.iterate(200)
    assert all(done)
    eb = B.energies()
    for s, inp, e in zip(specs, inps, eb):
        P = ccsd_k.Problem(s.grid, s.nocc, s.nvir, inp)
        ref = driver.solve(P, tol=1e-10, max_iter=200)
        assert abs(e.real - ref["energies"][-1].real / s.nk) < 1e-6
    B.close()


def test_mixed_batch_complex64_members(lib):
    """The batched workload's mixed members hold complex64 integrals: the same
    energies to 1e-6 Ha against the oracle on the widened integrals."""
    from paper_1911_00242_gb300.binding import CCSD_MIXED, BatchSolver
    specs = [cs.SynthSpec(**{**s.__dict__, "int_dtype": "c64"}) for s in (SPECS[0], SPECS[2], SPECS[3])]
    inps = [cs.generate(s) for s in specs]
    B = BatchSolver([(s.grid, s.nocc, s.nvir, dev(i)) for s, i in zip(specs, inps)], conv_tol=1e-7,
                    precision=CCSD_MIXED)
    done, mr = B.iterate(200)
    assert all(done)
    eb = B.energies()
    for s, inp, e in zip(specs, inps, eb):
        P = ccsd_k.Problem(s.grid, s.nocc, s.nvir, {k: np.asarray(v, np.complex128) for k, v in inp.items()})
        ref = driver.solve(P, tol=1e-10, max_iter=200)
        assert abs(e.real - ref["energies"][-1].real / s.nk) < 1e-6
    B.close()


def test_batch_diis_members_match_standalone(lib):
    """DIIS(6) inside the batch (grouped launches of the device-resident history, Gram
    matrix and Pulay solve) against each member run alone: energies after 6
    extrapolated updates within 1e-11 Ha."""
    from paper_1911_00242_gb300.binding import BatchSolver, Solver
    specs = SPECS[:4]
    inps = [cs.generate(s) for s in specs]
    devs = [dev(i) for i in inps]
    B = BatchSolver([(s.grid, s.nocc, s.nvir, d) for s, d in zip(specs, devs)], conv_tol=1e-30, diis_depth=6)
    B.iterate(6)
    eb = B.energies()
    for s, d, e in zip(specs, devs, eb):
        S = Solver(s.grid, s.nocc, s.nvir, d, conv_tol=1e-30, diis_depth=6)
        S.iterate(6)
        assert abs(S.energy() - e) < 1e-11, (s, S.energy(), e)
        S.close()
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_diis_converges_to_oracle(lib, precision):
    """Members with DIIS(6) converge to the oracle's DIIS(6) energies: FP64 members
    to 1e-8 Ha, mixed members (no polish inside the batch) to 1e-6 Ha."""
    from paper_1911_00242_gb300.binding import BatchSolver
    specs = SPECS[:4]
    inps = [cs.generate(s) for s in specs]
    B = BatchSolver([(s.grid, s.nocc, s.nvir, dev(i)) for s, i in zip(specs, inps)], conv_tol=1e-9 if precision == 0
                    else 1e-7, diis_depth=6, precision=precision)
    done, mr = B.iterate(100)
    assert all(done), (done, mr)
    eb = B.energies()
    for s, inp, e in zip(specs, inps, eb):
        P = ccsd_k.Problem(s.grid, s.nocc, s.nvir, inp)
        ref = driver.solve(P, tol=1e-10, max_iter=200, diis_depth=6)
        assert abs(e.real - ref["energies"][-1].real / s.nk) < (1e-8 if precision == 0 else 1e-6)
    B.close()
