"""Planted mistakes in the oracle (on the CPU) are caught by the pins.

Each case monkeypatches one plausible slip into the form-A oracle -- a dropped
term, a wrong factor, a missing conjugate, a wrong momentum label -- and checks
that the two-electron FCI pin or the unfolded-supercell pin sees it.  Slips in
form B -- the literal sign of Eq. def_F_oo, a dropped part of Eq. EqDouble -- are
caught by form A = form B."""
import numpy as np
import pytest

import ccsd_synth as cs
from helpers import dense_bloch, from_dense, to_dense
from oracle import ccsd_k, driver, fci, molecular


def _unfold_gap(spec):
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    Vk, fk, occ, vir = dense_bloch(spec)
    M = molecular.Dense(fk, Vk, occ, vir)
    t1, t2 = cs.random_amplitudes(spec, 5)
    D1, D2 = driver.denominators(P)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    T1, T2 = molecular.step(M, *to_dense(spec, t1, t2))
    k1, k2 = from_dense(spec, T1, T2)
    return max(abs(t1 + R1 / D1 - k1).max(), abs(t2 + R2 / D2 - k2).max())


def _fci_gap(spec):
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    r = driver.solve(P, tol=1e-12, max_iter=300)
    Vk, fk, occ, vir = dense_bloch(spec)
    return abs(r["energies"][-1] - fci.correlation_energy(fk, Vk, occ))


SPEC_U = cs.SynthSpec((2, 1, 1), 2, 3, 41, time_reversal=False, fock_offdiag=0.05)
SPEC_F = cs.SynthSpec((1, 1, 1), 2, 4, 21, time_reversal=False, fock_offdiag=0.1)


def test_unmutated_baseline():
    assert _unfold_gap(SPEC_U) < 1e-13
    assert _fci_gap(SPEC_F) < 1e-10


def _wrap(name, fn):
    orig = getattr(ccsd_k, name)
    def w(*a, **k):
        return fn(orig(*a, **k))
    return w


MUTATIONS = {
    # ladder coefficient 1/4 instead of 1/2 (W~^abef scaled by 1/2)
    "ladder_factor": ("w_abef", lambda W: 0.5 * W),
    # hole-hole intermediate without its oooo term is too drastic; drop its sign instead
    "w_mnij_sign": ("w_mnij", lambda W: -W),
    # ring intermediate transposed in (b, f)
    "ring_transposed": ("w_ring", lambda W: W.transpose(0, 1, 2, 3, 4, 6, 5).copy()),
    # F~_ov without its conjugate symmetry partner: conjugated by mistake
    "f_ov_conj": ("f_ov_tilde", lambda F: np.conj(F)),
    # tau~ used where tau belongs (t1 t1 factor 1/2 instead of 1)
    "tau_factor": ("taus", lambda tt: (tt[0], tt[0])),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    fn_name, mut = MUTATIONS[name]
    monkeypatch.setattr(ccsd_k, fn_name, _wrap(fn_name, mut))
    gaps = [_unfold_gap(SPEC_U)]
    try:
        gaps.append(_fci_gap(SPEC_F))
    except (np.linalg.LinAlgError, FloatingPointError):
        gaps.append(np.inf)
    assert max(gaps) > 1e-8, gaps


def test_missing_t1_driver_conjugate_is_caught(monkeypatch):
    orig = ccsd_k.residual
    def mutated(P, t1, t2):
        R1, R2 = orig(P, t1, t2)
        return R1 - np.conj(P.f_ov) + P.f_ov, R2
    monkeypatch.setattr(ccsd_k, "residual", mutated)
    spec = SPEC_F
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    r = driver.solve(P, residual=mutated, tol=1e-12, max_iter=300)
    Vk, fk, occ, vir = dense_bloch(spec)
    assert abs(r["energies"][-1] - fci.correlation_energy(fk, Vk, occ)) > 1e-8


def test_wrong_momentum_label_is_caught(monkeypatch):
    """vvvo block read at (kb, ka, ki) instead of (ka, kb, ki)."""
    orig_get = ccsd_k.Integrals.get
    def get(self, cls, kp, kq, kr):
        if cls == "vvvo" and kp != kq:
            return orig_get(self, cls, kq, kp, kr)
        return orig_get(self, cls, kp, kq, kr)
    monkeypatch.setattr(ccsd_k.Integrals, "get", get)
    spec = cs.SynthSpec((3, 1, 1), 2, 3, 44, time_reversal=False)
    assert _unfold_gap(spec) > 1e-8


# ---------------------------------------------------------------- form B readings
def _form_gap(spec):
    """max |R(form A) - R(form B)| on random amplitudes."""
    from oracle import ccsd_k_rearranged as form_b
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    t1, t2 = cs.random_amplitudes(spec, 6)
    a1, a2 = ccsd_k.residual(P, t1, t2)
    b1, b2 = form_b.residual(P, t1, t2)
    return max(abs(a1 - b1).max(), abs(a2 - b2).max())


SPEC_B = cs.SynthSpec((2, 2, 1), 2, 3, 47, time_reversal=False, fock_offdiag=0.05)


def test_form_b_baseline():
    assert _form_gap(SPEC_B) < 1e-12


def test_f_oo_sign_reading_is_pinned(monkeypatch):
    """Reading G1: Eq. def_F_oo taken literally, with (f - K~) in its t1 term instead of
    (f + K~), breaks form A = form B."""
    from oracle import ccsd_k_rearranged as form_b
    orig = form_b.fock_tilde

    def literal(P, t1, t2):
        Foo, Fvv, Fov = orig(P, t1, t2)
        K = form_b._k_tilde(P, t1)
        Foo = Foo.copy()
        for k in P.km:
            Foo[k] -= np.einsum("qc,pc->pq", t1[k], K[k])     # 1/2 t1 (f + K~) -> 1/2 t1 (f - K~)
        return Foo, Fvv, Fov

    monkeypatch.setattr(form_b, "fock_tilde", literal)
    assert _form_gap(SPEC_B) > 1e-8


@pytest.mark.parametrize("part", ["a_bar", "a_check", "a_tilde", "a_hat"])
def test_each_part_of_eq_double_is_pinned(monkeypatch, part):
    """Dropping any of the four parts of Eq. EqDouble breaks form A = form B."""
    from oracle import ccsd_k_rearranged as form_b
    orig = getattr(form_b, part)
    monkeypatch.setattr(form_b, part, lambda *a: 0.0 * orig(*a))
    assert _form_gap(SPEC_B) > 1e-8
