"""Checkpoint/resume through ccsd_get_amplitudes / ccsd_set_amplitudes, and the
per-step tracing API (ccsd_trace_*)."""
import numpy as np
import pytest

import ccsd_synth as cs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def test_resume_from_checkpoint_continues_the_iteration(lib):
    """3 updates, checkpoint, a new handle resumes for 2 more: the same amplitudes and
    energy as 5 uninterrupted updates (successive substitution carries no history)."""
    from paper_1911_00242_gb300.binding import Solver
    spec = cs.SynthSpec((3, 1, 1), 3, 5, 601)
    arrays = {k: dev(v) for k, v in cs.generate(spec).items()}
    A = Solver(spec.grid, spec.nocc, spec.nvir, arrays, conv_tol=1e-30)
    A.iterate(5)
    shape2 = (spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2
    B = Solver(spec.grid, spec.nocc, spec.nvir, arrays, conv_tol=1e-30)
    B.iterate(3)
    h1 = np.empty((spec.nk, spec.nocc, spec.nvir), np.complex128)
    h2 = np.empty(shape2, np.complex128)
    B.get_amplitudes(h1, h2)                       # checkpoint to host memory
    B.close()
    C = Solver(spec.grid, spec.nocc, spec.nvir, arrays, conv_tol=1e-30)
    C.set_amplitudes(h1, h2)                       # resume
    C.iterate(2)
    a1, a2 = torch.empty(h1.shape, dtype=torch.complex128, device="cuda"), torch.empty(shape2, dtype=torch.complex128, device="cuda")
    c1, c2 = torch.empty_like(a1), torch.empty_like(a2)
    A.get_amplitudes(a1, a2)
    C.get_amplitudes(c1, c2)
    assert torch.equal(a1, c1) and torch.equal(a2, c2)
    assert A.energy() == C.energy()


def test_trace_reports_every_step(lib):
    from paper_1911_00242_gb300.binding import Solver
    spec = cs.SynthSpec((2, 2, 1), 3, 6, 602)
    arrays = {k: dev(v) for k, v in cs.generate(spec).items()}
    S = Solver(spec.grid, spec.nocc, spec.nvir, arrays, conv_tol=1e-30)
    S.iterate(1)
    S.trace(True)
    S.iterate(2)
    steps = S.trace_steps()
    names = {s[0] for s in steps}
    for n in ("tau", "F_oo", "F_vv", "R1", "hole_hole", "ladder", "ring_W_t2", "ring", "antisym_R2", "update"):
        assert n in names, n
    ran = [s for s in steps if s[1] > 0]
    assert all(s[1] == 2 for s in ran)             # every active step ran once per iteration
    assert all(s[2] > 0 for s in ran)
    # the ring GEMMs' algorithmic flops: 8 N^4 o^3 v^3 each
    N, o, v = spec.nk, spec.nocc, spec.nvir
    ring = [s for s in ran if s[0] == "ring" and s[3] > 0]
    assert any(abs(s[3] - 8.0 * N ** 4 * o ** 3 * v ** 3) < 1 for s in ring)
    S.trace(False)
    S.close()
