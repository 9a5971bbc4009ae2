"""ccsd_energy_noalloc: the correlation energy without device allocation.

It serves callers that cannot call cudaMalloc (inside a stream capture, under
an allocator that owns all device memory, or in allocation-free loops).  This
file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import ccsd_synth as cs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dims(grid):
    return (ctypes.c_int * 3)(*grid)


def test_noalloc_energy_matches_handle_energy(lib):
    from paper_1911_00242_gb300.binding import Solver
    spec = cs.SynthSpec((3, 2, 1), 3, 5, 901, time_reversal=False, fock_offdiag=0.05)
    inp = cs.generate(spec)
    dev = {k: torch.from_numpy(v).to("cuda") for k, v in inp.items()}
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev)
    t1 = torch.empty((spec.nk, spec.nocc, spec.nvir), dtype=torch.complex128, device="cuda")
    t2 = torch.empty((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, dtype=torch.complex128, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for n_iter in (2, 1):       # two calls in a row, on different amplitudes
        S.iterate(n_iter)
        ref = S.energy()
        S.get_amplitudes(t1, t2)
        rc = lib.ccsd_energy_noalloc(_dims(spec.grid), spec.nocc, spec.nvir, dev["f_ov"].data_ptr(),
                                     dev["oovv"].data_ptr(), t1.data_ptr(), t2.data_ptr(), out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        e = out.cpu().numpy()
        assert abs(e[0] - ref.real) < 1e-12 and abs(e[1] - ref.imag) < 1e-12, (e, ref)
    S.close()


def test_noalloc_rejects_grids_beyond_its_scratch(lib):
    buf = torch.zeros(16, dtype=torch.complex128, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    # 32 k points need 32^3 + 1 = 32769 partial sums: one more than the 32768 the library holds
    rc = lib.ccsd_energy_noalloc(_dims((32, 1, 1)), 2, 3, p, p, p, p, out.data_ptr(), None)
    assert rc == -1
    # grid sides beyond 64 are refused before N_k^3 is formed (it would overflow 64 bits)
    for grid in ((65, 1, 1), (1 << 21, 1, 1), (1 << 21, 1 << 21, 1 << 21)):
        assert lib.ccsd_energy_noalloc(_dims(grid), 2, 3, p, p, p, p, out.data_ptr(), None) == -1
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0)
