"""k-free spin-orbital CCSD on dense tensors (the molecular limit).

Written in the textbook Jacobi form of Stanton, Gauss, Watts and Bartlett
(J. Chem. Phys. 94, 4334 (1991)) on which the paper's Eqs. ori_EqSingle and
ori_EqDouble build: the Fock diagonal is removed from F and each step is
t_new = RHS / D.  With complex orbitals the doubles driver is <ab||ij> and the
singles driver <a|f|i>.  It takes the full antisymmetrized tensor
V[p, q, r, s] = <pq||rs> and the Fock matrix in any orthonormal spin-orbital
basis, with explicit lists of occupied and virtual orbitals, and knows nothing
about momenta.  Used to pin the k-point oracle at N_k = 1 and on the unfolded
supercell.
"""
import numpy as np

def ein(*args):
    # BLAS-backed einsum (numpy picks the pairwise contraction order)
    return np.einsum(*args, optimize=True)


class Dense:
    def __init__(self, f, V, occ, vir):
        self.o = np.asarray(occ)
        self.v = np.asarray(vir)
        self.f = np.asarray(f, np.complex128)
        self.V = np.asarray(V, np.complex128)

    def blk(self, cls):
        sel = {"o": self.o, "v": self.v}
        return self.V[np.ix_(*(sel[c] for c in cls))]

    def fblk(self, cls):
        sel = {"o": self.o, "v": self.v}
        return self.f[np.ix_(sel[cls[0]], sel[cls[1]])]


def _pij(X):
    return X - X.transpose(1, 0, 2, 3)


def _pab(X):
    return X - X.transpose(0, 1, 3, 2)


def step(M: Dense, t1, t2):
    """One Jacobi step: returns (t1_new, t2_new)."""
    foo, fvv, fov = M.fblk("oo"), M.fblk("vv"), M.fblk("ov")
    Do = np.diag(foo).real
    Dv = np.diag(fvv).real
    D1 = Do[:, None] - Dv[None, :]
    D2 = Do[:, None, None, None] + Do[None, :, None, None] - Dv[None, None, :, None] - Dv[None, None, None, :]
    foo_d = foo - np.diag(np.diag(foo))
    fvv_d = fvv - np.diag(np.diag(fvv))
    oovv, ooov, ovvv = M.blk("oovv"), M.blk("ooov"), M.blk("ovvv")
    tt = ein("ia,jb->ijab", t1, t1) - ein("ib,ja->ijab", t1, t1)
    taut = t2 + 0.5 * tt
    tau = t2 + tt

    Fae = fvv_d - 0.5 * ein("me,ma->ae", fov, t1) + ein("mf,mafe->ae", t1, ovvv) \
        - 0.5 * ein("mnaf,mnef->ae", taut, oovv)
    Fmi = foo_d + 0.5 * ein("ie,me->mi", t1, fov) + ein("ne,mnie->mi", t1, ooov) \
        + 0.5 * ein("inef,mnef->mi", taut, oovv)
    Fme = fov + ein("nf,mnef->me", t1, oovv)

    X = ein("je,mnie->mnij", t1, ooov)
    Wmnij = M.blk("oooo") + X - X.transpose(0, 1, 3, 2) + 0.25 * ein("ijef,mnef->mnij", tau, oovv)
    Y = ein("mb,amef->abef", t1, M.blk("vovv"))
    Wabef = M.blk("vvvv") - (Y - Y.transpose(1, 0, 2, 3)) + 0.25 * ein("mnab,mnef->abef", tau, oovv)
    Wmbej = M.blk("ovvo") + ein("jf,mbef->mbej", t1, ovvv) - ein("nb,mnej->mbej", t1, M.blk("oovo")) \
        - ein("jnfb,mnef->mbej", 0.5 * t2, oovv) - ein("jf,nb,mnef->mbej", t1, t1, oovv)

    r1 = np.conj(fov) + ein("ie,ae->ia", t1, Fae) - ein("ma,mi->ia", t1, Fmi) \
        + ein("imae,me->ia", t2, Fme) - ein("nf,naif->ia", t1, M.blk("ovov")) \
        - 0.5 * ein("imef,maef->ia", t2, ovvv) - 0.5 * ein("mnae,nmei->ia", t2, M.blk("oovo"))

    r2 = M.blk("vvoo").transpose(2, 3, 0, 1).copy()
    r2 += _pab(ein("ijae,be->ijab", t2, Fae - 0.5 * ein("mb,me->be", t1, Fme)))
    r2 -= _pij(ein("imab,mj->ijab", t2, Fmi + 0.5 * ein("je,me->mj", t1, Fme)))
    r2 += 0.5 * ein("mnab,mnij->ijab", tau, Wmnij)
    r2 += 0.5 * ein("ijef,abef->ijab", tau, Wabef)
    r2 += _pij(_pab(ein("imae,mbej->ijab", t2, Wmbej) - ein("ie,ma,mbej->ijab", t1, t1, M.blk("ovvo"))))
    r2 += _pij(ein("ie,abej->ijab", t1, M.blk("vvvo")))
    r2 -= _pab(ein("ma,mbij->ijab", t1, M.blk("ovoo")))
    return r1 / D1, r2 / D2


def energy(M: Dense, t1, t2):
    oovv = M.blk("oovv")
    return ein("ia,ia->", M.fblk("ov"), t1) + 0.25 * ein("ijab,ijab->", oovv, t2) \
        + 0.5 * ein("ijab,ia,jb->", oovv, t1, t1)


def solve(M: Dense, tol=1e-10, max_iter=200):
    """Jacobi iterations from t = 0 until max|t_new - t| < tol; returns (E, t1, t2, n)."""
    no, nv = len(M.o), len(M.v)
    t1 = np.zeros((no, nv), np.complex128)
    t2 = np.zeros((no, no, nv, nv), np.complex128)
    for it in range(1, max_iter + 1):
        n1, n2 = step(M, t1, t2)
        d = max(abs(n1 - t1).max(initial=0.0), abs(n2 - t2).max(initial=0.0))
        t1, t2 = n1, n2
        if d < tol:
            return energy(M, t1, t2), t1, t2, it
    raise RuntimeError("molecular CCSD did not converge")
