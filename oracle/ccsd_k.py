"""Form A: the original periodic CCSD equations (paper Sec. 2).

T1 residual: Eq. (ori_EqSingle); T2 residual: Eq. (ori_EqDouble); the
intermediates W~_mnij, W~^abef, W~_jn^bf (Eq. Def_Woovv), F~ (Eqs. ori_F_oo,
ori_F_vv, ori_F_ov) and the effective doubles tau~, tau.

Arrays (complex128):
  t1[k, i, a];  t2[ki, kj, ka, i, j, a, b] with kb = ki + kj - ka
  f_oo[k, i, j], f_vv[k, a, b], f_ov[k, i, a]
Every sum runs over all orbital indices and all independent momenta; the
dependent momentum follows from conservation (Sec. 3.2.5).  The residual R is
the right-hand side of the paper's equations written as 0 = R, with the full
Fock matrix inside F~ (no diagonal removed), as the paper states it.
"""
import numpy as np

from .integrals import Integrals
from .kmesh import KMesh

def ein(*args):
    # BLAS-backed einsum (numpy picks the pairwise contraction order)
    return np.einsum(*args, optimize=True)


class Problem:
    """Inputs of one periodic CCSD problem."""

    def __init__(self, grid, nocc, nvir, arrays: dict):
        self.km = KMesh(grid)
        self.nk, self.o, self.v = self.km.nk, nocc, nvir
        self.f_oo = np.asarray(arrays["f_oo"], np.complex128)
        self.f_vv = np.asarray(arrays["f_vv"], np.complex128)
        self.f_ov = np.asarray(arrays["f_ov"], np.complex128)
        blocks = {k: np.asarray(arrays[k], np.complex128) for k in Integrals.STORED}
        self.I = Integrals(blocks, self.km)


def taus(P: Problem, t1, t2):
    """tau~ = t2 + 1/4 P(ab)P(ij) t1 t1 and tau = t2 + 1/2 P(ab)P(ij) t1 t1.

    t_{i ki}^{a ka} t_{j kj}^{b kb} is non-zero only for ki = ka (then kj = kb);
    the four terms of P(ab)P(ij) pair up, so 1/2 P(ab)P(ij) t t equals
    delta(ki,ka) t_i^a t_j^b - delta(ki,kb) t_i^b t_j^a."""
    km = P.km
    tau_t = t2.copy()
    tau = t2.copy()
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                x = np.zeros(t2.shape[3:], np.complex128)
                if ki == ka:
                    x += ein("ia,jb->ijab", t1[ki], t1[kj])
                if ki == kb:
                    x -= ein("ib,ja->ijab", t1[ki], t1[kj])
                tau_t[ki, kj, ka] += 0.5 * x
                tau[ki, kj, ka] += x
    return tau_t, tau


def f_ov_tilde(P: Problem, t1):
    """F~_p^g(k) = f_p^g + sum_{r c k^} t_r^c(k^) <p k r k^||g k c k^>   (Eq. ori_F_ov)."""
    km, I = P.km, P.I
    F = P.f_ov.copy()
    for k in km:
        for kh in km:
            F[k] += ein("rc,prgc->pg", t1[kh], I.get("oovv", k, kh, k))
    return F


def f_oo_tilde(P: Problem, t1, tau_t):
    """F~_pq(k)   (Eq. ori_F_oo)."""
    km, I = P.km, P.I
    F = P.f_oo.copy()
    for k in km:
        F[k] += 0.5 * ein("pc,qc->pq", P.f_ov[k], t1[k])
        for kh in km:
            F[k] += ein("rc,prqc->pq", t1[kh], I.get("ooov", k, kh, k))
        for kn in km:
            for ke in km:
                F[k] += 0.5 * ein("qnef,pnef->pq", tau_t[k, kn, ke], I.get("oovv", k, kn, ke))
    return F


def f_vv_tilde(P: Problem, t1, tau_t):
    """F~^gh(k)   (Eq. ori_F_vv)."""
    km, I = P.km, P.I
    F = P.f_vv.copy()
    for k in km:
        F[k] -= 0.5 * ein("rh,rg->gh", P.f_ov[k], t1[k])
        for kh in km:
            F[k] += ein("rc,grhc->gh", t1[kh], I.get("vovv", k, kh, k))
        for kmm in km:
            for kn in km:
                F[k] -= 0.5 * ein("mngf,mnhf->gh", tau_t[kmm, kn, k], I.get("oovv", kmm, kn, k))
    return F


def w_mnij(P: Problem, t1, tau):
    """W~_{m km n kn i ki j kj}, stored [km, kn, ki, m, n, i, j]  (kj implied)."""
    km, I = P.km, P.I
    N, o = P.nk, P.o
    W = np.zeros((N, N, N, o, o, o, o), np.complex128)
    for kmm in km:
        for kn in km:
            for ki in km:
                kj = km.k4(kmm, kn, ki)
                w = I.get("oooo", kmm, kn, ki).copy()
                # P(ij) sum_c t_j^c <mn||ic>
                w += ein("jc,mnic->mnij", t1[kj], I.get("ooov", kmm, kn, ki))
                w -= ein("ic,mnjc->mnij", t1[ki], I.get("ooov", kmm, kn, kj))
                for ke in km:
                    w += 0.25 * ein("ijef,mnef->mnij", tau[ki, kj, ke], I.get("oovv", kmm, kn, ke))
                W[kmm, kn, ki] = w
    return W


def w_abef(P: Problem, t1, tau):
    """W~^{a ka b kb e ke f kf}, stored [ka, kb, ke, a, b, e, f]  (kf implied)."""
    km, I = P.km, P.I
    N, v = P.nk, P.v
    W = np.zeros((N, N, N, v, v, v, v), np.complex128)
    for ka in km:
        for kb in km:
            for ke in km:
                w = I.get("vvvv", ka, kb, ke).copy()
                # -P(ab) sum_r t_r^b <a r||e f>   (r carries kb, then ka)
                w -= ein("rb,aref->abef", t1[kb], I.get("vovv", ka, kb, ke))
                w += ein("ra,bref->abef", t1[ka], I.get("vovv", kb, ka, ke))
                for kmm in km:
                    kn = km.k4(ka, kb, kmm)
                    w += 0.25 * ein("mnab,mnef->abef", tau[kmm, kn, ka], I.get("oovv", kmm, kn, ke))
                W[ka, kb, ke] = w
    return W


def w_ring(P: Problem, t1, t2):
    """W~_{j kj n kn}^{b kb f kf}, stored [kj, kn, kb, j, n, b, f], kf = kn + kb - kj  (Eq. Def_Woovv)."""
    km, I = P.km, P.I
    N, o, v = P.nk, P.o, P.v
    W = np.zeros((N, N, N, o, o, v, v), np.complex128)
    for kj in km:
        for kn in km:
            for kb in km:
                kf = km.k4(kn, kb, kj)
                w = ein("nbfj->jnbf", I.get("ovvo", kn, kb, kf))
                w += ein("jc,nbfc->jnbf", t1[kj], I.get("ovvv", kn, kb, kf))
                w -= ein("rb,nrfj->jnbf", t1[kb], I.get("oovo", kn, kb, kf))
                for kx in km:
                    ky = km.k4(kj, kx, kb)
                    w -= 0.5 * ein("jxyb,nxfy->jnbf", t2[kj, kx, ky], I.get("oovv", kn, kx, kf))
                w -= ein("jc,rb,nrfc->jnbf", t1[kj], t1[kb], I.get("oovv", kn, kb, kf))
                W[kj, kn, kb] = w
    return W


def _pij(Z, km):
    """P(ij) Z over the t2 layout: Z[ki,kj,ka](ijab) - Z[kj,ki,ka](jiab)."""
    out = np.empty_like(Z)
    for ki in km:
        for kj in km:
            for ka in km:
                out[ki, kj, ka] = Z[ki, kj, ka] - Z[kj, ki, ka].transpose(1, 0, 2, 3)
    return out


def _pab(Z, km):
    """P(ab) Z over the t2 layout: Z[ki,kj,ka](ijab) - Z[ki,kj,kb](ijba)."""
    out = np.empty_like(Z)
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                out[ki, kj, ka] = Z[ki, kj, ka] - Z[ki, kj, kb].transpose(0, 1, 3, 2)
    return out


def residual(P: Problem, t1, t2):
    """(R1, R2) of form A at amplitudes (t1, t2)."""
    km, I = P.km, P.I
    N, o, v = P.nk, P.o, P.v
    tau_t, tau = taus(P, t1, t2)
    Fov = f_ov_tilde(P, t1)
    Foo = f_oo_tilde(P, t1, tau_t)
    Fvv = f_vv_tilde(P, t1, tau_t)

    # ---------------- T1 (Eq. ori_EqSingle)
    # driver f_p^g read as <g k|f|p k> = f_ov[k][p][g]^*; inside F~ it is <p|f|g>
    R1 = np.conj(P.f_ov).copy()
    for k in km:
        R1[k] += ein("ac,ic->ia", Fvv[k], t1[k])
        R1[k] -= ein("ra,ri->ia", t1[k], Foo[k])
        for kh in km:
            R1[k] += ein("nf,inaf->ia", Fov[kh], t2[k, kh, k])
            R1[k] += ein("rc,aric->ia", t1[kh], I.get("voov", k, kh, k))
        for kmm in km:
            for kn in km:
                R1[k] -= 0.5 * ein("mnaf,mnif->ia", t2[kmm, kn, k], I.get("ooov", kmm, kn, k))
        for kn in km:
            for ke in km:
                R1[k] += 0.5 * ein("inef,anef->ia", t2[k, kn, ke], I.get("vovv", k, kn, ke))

    # ---------------- T2 (Eq. ori_EqDouble)
    Wmnij = w_mnij(P, t1, tau)
    Wabef = w_abef(P, t1, tau)
    Wring = w_ring(P, t1, t2)
    Fvv_p = np.empty_like(Fvv)   # F~^bf - 1/2 sum_r t_r^b F~_r^f
    Foo_p = np.empty_like(Foo)   # F~_nj + 1/2 sum_c t_j^c F~_n^c
    for k in km:
        Fvv_p[k] = Fvv[k] - 0.5 * ein("rb,rf->bf", t1[k], Fov[k])
        Foo_p[k] = Foo[k] + 0.5 * ein("jc,nc->nj", t1[k], Fov[k])

    R2 = np.zeros_like(t2)
    Zab = np.zeros_like(t2)     # terms under P(ab)
    Zij = np.zeros_like(t2)     # terms under P(ij)
    Zijab = np.zeros_like(t2)   # terms under P(ij) P(ab)
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                r = np.conj(I.get("oovv", ki, kj, ka))             # <ab||ij> = <ij||ab>^*
                Zab[ki, kj, ka] += ein("ijaf,bf->ijab", t2[ki, kj, ka], Fvv_p[kb])
                Zij[ki, kj, ka] -= ein("inab,nj->ijab", t2[ki, kj, ka], Foo_p[kj])
                for kmm in km:
                    kn = km.k4(ki, kj, kmm)
                    r += 0.5 * ein("mnab,mnij->ijab", tau[kmm, kn, ka], Wmnij[kmm, kn, ki])
                for ke in km:
                    r += 0.5 * ein("abef,ijef->ijab", Wabef[ka, kb, ke], tau[ki, kj, ke])
                for kn in km:
                    Zijab[ki, kj, ka] += ein("inaf,jnbf->ijab", t2[ki, kn, ka], Wring[kj, kn, kb])
                Zijab[ki, kj, ka] -= ein("ic,ra,rbcj->ijab", t1[ki], t1[ka],
                                         I.get("ovvo", ka, kb, ki))
                Zij[ki, kj, ka] += ein("abcj,ic->ijab", I.get("vvvo", ka, kb, ki), t1[ki])
                Zab[ki, kj, ka] -= ein("ra,rbij->ijab", t1[ka], I.get("ovoo", ka, kb, ki))
                R2[ki, kj, ka] = r
    R2 += _pab(Zab, km) + _pij(Zij, km) + _pij(_pab(Zijab, km), km)
    return R1, R2


def energy(P: Problem, t1, t2):
    """Total (supercell) correlation energy, complex:
    sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b.
    The paper gives no energy expression; this is the standard one."""
    km, I = P.km, P.I
    e = 0j
    for k in km:
        e += ein("ia,ia->", P.f_ov[k], t1[k])
    for ki in km:
        for kj in km:
            for ka in km:
                e += 0.25 * ein("ijab,ijab->", I.get("oovv", ki, kj, ka), t2[ki, kj, ka])
            e += 0.5 * ein("ijab,ia,jb->", I.get("oovv", ki, kj, ki), t1[ki], t1[kj])
    return e
