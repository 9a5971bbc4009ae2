"""Full CI for two electrons: CCSD is exact there.

Given f and V = <pq||rs> over M spin orbitals and the occupied pair (i0, j0)
of the reference, the core Hamiltonian is h = f - sum_m <pm||qm> over the
occupied m.  Determinants |pq> = p^+ q^+ |0> (p < q) span the space; their
Hamiltonian matrix is
  <pq|H|rs> = h_pr d_qs - h_ps d_qr - h_qr d_ps + h_qs d_pr + <pq||rs>,
and the reference energy is E_ref = sum_i h_ii + 1/2 sum_ij <ij||ij>.
"""
import numpy as np


def correlation_energy(f, V, occ):
    occ = list(occ)
    assert len(occ) == 2
    M = f.shape[0]
    h = f - np.einsum("pmqm->pq", V[:, occ][:, :, :, occ])
    dets = [(p, q) for p in range(M) for q in range(p + 1, M)]
    n = len(dets)
    H = np.zeros((n, n), np.complex128)
    for x, (p, q) in enumerate(dets):
        for y, (r, s) in enumerate(dets):
            e = V[p, q, r, s]
            if q == s:
                e += h[p, r]
            if q == r:
                e -= h[p, s]
            if p == s:
                e -= h[q, r]
            if p == r:
                e += h[q, s]
            H[x, y] = e
    w = np.linalg.eigvalsh(H)
    e_ref = sum(h[i, i] for i in occ) + 0.5 * sum(V[i, j, i, j] for i in occ for j in occ)
    return w[0] - e_ref.real
