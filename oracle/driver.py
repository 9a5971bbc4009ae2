"""Iteration driver (paper Sec. 4.1 and Sec. 4.4), DIIS and energy.

* start: t0 = f(0), i.e. one update from t = 0 (Sec. 3.2.2);
* update: t <- t + R / D with D_i^a = f_ii - f^aa and
  D_ij^ab = f_ii + f_jj - f^aa - f^bb (Eqs. in Sec. 4.4.19);
* stop when max|R1| < eps and max|R2| < eps (Eqs. criterion_single/double);
* optional DIIS (not in the paper, which uses plain successive substitution):
  Pulay extrapolation over the last m updates with error vectors e = R / D,
  B_ij = Re <e_i|e_j>, coefficients summing to one.
"""
import numpy as np

from . import ccsd_k


def denominators(P):
    eo = np.real(np.einsum("kii->ki", P.f_oo))
    ev = np.real(np.einsum("kaa->ka", P.f_vv))
    km = P.km
    N = P.nk
    D1 = eo[:, :, None] - ev[:, None, :]
    D2 = np.empty((N, N, N, P.o, P.o, P.v, P.v))
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                D2[ki, kj, ka] = (eo[ki][:, None, None, None] + eo[kj][None, :, None, None]
                                  - ev[ka][None, None, :, None] - ev[kb][None, None, None, :])
    return D1, D2


class DIIS:
    def __init__(self, depth):
        self.depth = depth
        self.x, self.e = [], []

    def update(self, x, e):
        self.x.append(x)
        self.e.append(e)
        if len(self.x) > self.depth:
            self.x.pop(0)
            self.e.pop(0)
        m = len(self.x)
        if m < 2:
            return x
        B = np.zeros((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                B[i, j] = np.real(np.vdot(self.e[i], self.e[j]))
        B[m, :m] = B[:m, m] = -1.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.solve(B, rhs)[:m]
        return sum(ci * xi for ci, xi in zip(c, self.x))


def solve(P, residual=ccsd_k.residual, tol=1e-8, max_iter=100, diis_depth=0,
          n_iter=None, callback=None):
    """Iterate from t = 0.  Returns dict(t1, t2, energies, max_r, converged, iters).

    energies[n] is the energy after update n (energies[0] is E(t0) = MP2 when
    f_ov = 0).  With n_iter set, exactly n_iter updates are made."""
    N, o, v = P.nk, P.o, P.v
    t1 = np.zeros((N, o, v), np.complex128)
    t2 = np.zeros((N, N, N, o, o, v, v), np.complex128)
    D1, D2 = denominators(P)
    diis = DIIS(diis_depth) if diis_depth else None
    energies, max_r = [], []
    converged = False
    it = 0
    while True:
        R1, R2 = residual(P, t1, t2)
        mr = max(abs(R1).max(initial=0.0), abs(R2).max(initial=0.0))
        if it > 0:
            max_r.append(mr)
            if n_iter is None and mr < tol:
                converged = True
                break
        if (n_iter is not None and it >= n_iter) or it >= max_iter:
            break
        n1 = t1 + R1 / D1
        n2 = t2 + R2 / D2
        if diis is not None:
            x = np.concatenate([n1.ravel(), n2.ravel()])
            e = np.concatenate([(R1 / D1).ravel(), (R2 / D2).ravel()])
            x = diis.update(x, e)
            n1 = x[:n1.size].reshape(n1.shape)
            n2 = x[n1.size:].reshape(n2.shape)
        t1, t2 = n1, n2
        it += 1
        energies.append(ccsd_k.energy(P, t1, t2))
        if callback is not None:
            callback(it, t1, t2, energies[-1])
    return dict(t1=t1, t2=t2, energies=energies, max_r=max_r, converged=converged, iters=it)
