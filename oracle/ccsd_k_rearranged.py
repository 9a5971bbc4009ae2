"""Form B: the rearranged periodic CCSD equations (paper Sec. 3.3).

Intermediates rho-check/rho-hat (Sec. 3.3.1) are t1 itself on one process.
F~ through K~ and Z~ (Eqs. def_F_oo, def_F_vv, def_F_ov, def_Z_oo, def_Z_vv,
def_K); T1 through L~ (Eqs. EqSingle, def_L_oo, def_L_vv); T2 as the sum of
the four parts of Eq. EqDouble:
  A-bar   (Eq. A_1st with def_zeta, def_C, rearranged_W, def_J)
  A-check (Eq. A_2nd with eta, G-check, def_Y_vv and V~^abef)
  A-tilde (Eqs. A_3rd, def_X)
  A-hat   (Eq. A_4th with eta, G-hat, def_Y_oo and V~_mnij)

Readings where the text is garbled (each checked against form A):
  * def_F_oo: the t1 (f - K~) factor is read as (f + K~), which is what
    expanding tau~ in Eq. ori_F_oo gives and what def_F_vv has.
  * A_1st: zeta~_ri^ac is the product t_{r ka}^{a ka} t_{i ki}^{c ki}
    (momenta in the order that conserves momentum with the integral).
  * The T1 driver f_p^g is read as <g k|f|p k> = (f_ov[k][p][g])^*, while
    f_p^g inside F~ is <p k|f|g k>; the two agree for real orbitals.
"""
import numpy as np

from .ccsd_k import Problem  # noqa: F401  (same input container)

def ein(*args):
    # BLAS-backed einsum (numpy picks the pairwise contraction order)
    return np.einsum(*args, optimize=True)


def _k_tilde(P, t1):
    """K~_x^y(k) = sum_{r c k^} t_r^c(k^) <x k r k^||y k c k^>   (Eq. def_K)."""
    km, I = P.km, P.I
    K = np.zeros_like(P.f_ov)
    for k in km:
        for kh in km:
            K[k] += ein("rc,xryc->xy", t1[kh], I.get("oovv", k, kh, k))
    return K


def fock_tilde(P, t1, t2):
    """(F~_oo, F~_vv, F~_ov)   (Eqs. def_F_oo, def_F_vv, def_F_ov)."""
    km, I = P.km, P.I
    K = _k_tilde(P, t1)
    Foo = P.f_oo.copy()
    Fvv = P.f_vv.copy()
    for k in km:
        Foo[k] += 0.5 * ein("qc,pc->pq", t1[k], P.f_ov[k] + K[k])
        Fvv[k] -= 0.5 * ein("rg,rh->gh", t1[k], P.f_ov[k] + K[k])
        for kh in km:
            Foo[k] += ein("rc,prqc->pq", t1[kh], I.get("ooov", k, kh, k))
            Fvv[k] += ein("rc,rgch->gh", t1[kh], I.get("ovvv", kh, k, kh))
        for ke in km:                        # sum_{ke} Z~_pq^{ke}
            z = np.zeros((P.o, P.o), np.complex128)
            for kn in km:
                z += 0.5 * ein("qnef,pnef->pq", t2[k, kn, ke], I.get("oovv", k, kn, ke))
            Foo[k] += z
        for kmm in km:                       # - sum_{km} Z~_{km}^gh
            z = np.zeros((P.v, P.v), np.complex128)
            for kn in km:
                z += 0.5 * ein("mngf,mnhf->gh", t2[kmm, kn, k], I.get("oovv", kmm, kn, k))
            Fvv[k] -= z
    Fov = P.f_ov + K
    return Foo, Fvv, Fov


def residual_t1(P, t1, t2, Foo, Fvv, Fov):
    """R1 of Eq. EqSingle with the partial sums L~ (Eqs. def_L_oo, def_L_vv)."""
    km, I = P.km, P.I
    R1 = np.conj(P.f_ov).copy()
    for k in km:
        R1[k] += ein("pc,gc->pg", t1[k], Fvv[k])
        R1[k] -= ein("rg,rp->pg", t1[k], Foo[k])
        for kh in km:
            R1[k] += ein("pngf,nf->pg", t2[k, kh, k], Fov[kh])
            R1[k] += ein("rc,rgcp->pg", t1[kh], I.get("ovvo", kh, k, kh))
        for kmm in km:                        # - sum_{km} L~_{p, km}^g
            L = np.zeros((P.o, P.v), np.complex128)
            for kn in km:
                L += 0.5 * ein("mngf,mnpf->pg", t2[kmm, kn, k], I.get("ooov", kmm, kn, k))
            R1[k] -= L
        for ke in km:                         # + sum_{ke} L~_p^{g, ke}
            L = np.zeros((P.o, P.v), np.complex128)
            for kn in km:
                kf = km.k4(k, kn, ke)
                L += 0.5 * ein("pnef,ngfe->pg", t2[k, kn, ke], I.get("ovvv", kn, k, kf))
            R1[k] += L
    return R1


def a_bar(P, t1, t2):
    """A-bar = P(ij)P(ab) C~ + <ij||ab>^* + t1^4 term   (Eq. A_1st)."""
    km, I = P.km, P.I
    N, o, v = P.nk, P.o, P.v
    # W~_jn^bf, stored [kj, kn, kb](j, n, b, f), kf = kn + kb - kj  (Eqs. rearranged_W, def_J)
    W = np.zeros((N, N, N, o, o, v, v), np.complex128)
    for kj in km:
        for kn in km:
            for kb in km:
                kf = km.k4(kn, kb, kj)
                w = np.zeros((o, o, v, v), np.complex128)
                for ky in km:
                    kx = km.k4(kj, ky, kb)
                    w -= 0.5 * ein("jyxb,nyfx->jnbf", t2[kj, ky, kx], I.get("oovv", kn, ky, kf))
                w += ein("nbfj->jnbf", I.get("ovvo", kn, kb, kf))
                # J~
                w += ein("jc,nbfc->jnbf", t1[kj], I.get("ovvv", kn, kb, kf))
                w -= ein("rb,rnjf->jnbf", t1[kb], I.get("ooov", kb, kn, kj))
                w -= ein("rb,jc,rncf->jnbf", t1[kb], t1[kj], I.get("oovv", kb, kn, kj))
                W[kj, kn, kb] = w
    C = np.zeros_like(t2)
    out = np.zeros_like(t2)
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                c = np.zeros((o, o, v, v), np.complex128)
                for kn in km:
                    c += ein("inaf,jnbf->ijab", t2[ki, kn, ka], W[kj, kn, kb])
                c -= ein("rb,jc,raci->ijab", t1[kb], t1[kj], I.get("ovvo", kb, ka, kj))
                C[ki, kj, ka] = c
                out[ki, kj, ka] = np.conj(I.get("oovv", ki, kj, ka))
                out[ki, kj, ka] += ein("ra,sb,ic,jd,rscd->ijab", t1[ka], t1[kb], t1[ki], t1[kj],
                                       I.get("oovv", ka, kb, ki))
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                out[ki, kj, ka] += (C[ki, kj, ka]
                                    - C[kj, ki, ka].transpose(1, 0, 2, 3)
                                    - C[ki, kj, kb].transpose(0, 1, 3, 2)
                                    + C[kj, ki, kb].transpose(1, 0, 3, 2))
    return out


def a_check(P, t1, t2, Fvv, Fov):
    """A-check   (Eq. A_2nd with eta~, G-check, Y~^abef of Eq. def_Y_vv, V~^abef)."""
    km, I = P.km, P.I
    N, o, v = P.nk, P.o, P.v
    # V~^abef [ka, kb, ke](a, b, e, f) = sum_r t_r^b(kb) <r kb a ka||e ke f kf>
    Vt = np.zeros((N, N, N, v, v, v, v), np.complex128)
    for ka in km:
        for kb in km:
            for ke in km:
                Vt[ka, kb, ke] = ein("rb,raef->abef", t1[kb], I.get("ovvv", kb, ka, ke))
    Y = np.zeros_like(Vt)
    for ka in km:
        for kb in km:
            for ke in km:
                y = Vt[ka, kb, ke] - Vt[kb, ka, ke].transpose(1, 0, 2, 3)
                y -= I.get("vvvv", kb, ka, ke).transpose(1, 0, 2, 3)
                y -= ein("sb,ra,sref->abef", t1[kb], t1[ka], I.get("oovv", kb, ka, ke))
                Y[ka, kb, ke] = 0.5 * y
    G = np.zeros_like(t2)
    out = np.zeros_like(t2)
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                eta = ein("ra,sb->rsab", t1[ka], t1[kb])
                x = ein("rsab,rsij->ijab", eta, I.get("oooo", ka, kb, ki))
                g = ein("rsab,rsic->icab", eta, I.get("ooov", ka, kb, ki))
                g += np.conj(I.get("ovvv", ki, kj, ka))
                G[ki, kj, ka] = ein("jc,icab->ijab", t1[kj], g)
                fb = Fvv[kb] - 0.5 * ein("rb,rf->bf", t1[kb], Fov[kb])
                fa = Fvv[ka] - 0.5 * ein("ra,rf->af", t1[ka], Fov[ka])
                # P(ab) sum_f t_ij^{af} (F~^{bf} - 1/2 t_r^b F~_r^f)
                x += ein("ijaf,bf->ijab", t2[ki, kj, ka], fb)
                x -= ein("ijbf,af->ijab", t2[ki, kj, kb], fa)
                for ke in km:
                    x += ein("ijef,abef->ijab", t2[ki, kj, ke], Y[ka, kb, ke])
                out[ki, kj, ka] = x
    for ki in km:
        for kj in km:
            for ka in km:
                out[ki, kj, ka] += G[ki, kj, ka] - G[kj, ki, ka].transpose(1, 0, 2, 3)
    return out


def a_tilde(P, t1, t2):
    """A-tilde = 1/4 sum t_mn^ab X~_mnij, X~ = sum t_ij^ef <mn||ef>   (Eqs. A_3rd, def_X)."""
    km, I = P.km, P.I
    N, o = P.nk, P.o
    X = np.zeros((N, N, N, o, o, o, o), np.complex128)
    for kmm in km:
        for kn in km:
            for ki in km:
                kj = km.k4(kmm, kn, ki)
                for ke in km:
                    X[kmm, kn, ki] += ein("ijef,mnef->mnij", t2[ki, kj, ke], I.get("oovv", kmm, kn, ke))
    out = np.zeros_like(t2)
    for ki in km:
        for kj in km:
            for ka in km:
                for kmm in km:
                    kn = km.k4(ki, kj, kmm)
                    out[ki, kj, ka] += 0.25 * ein("mnab,mnij->ijab", t2[kmm, kn, ka], X[kmm, kn, ki])
    return out


def a_hat(P, t1, t2, Foo, Fov):
    """A-hat   (Eq. A_4th with eta~, G-hat, Y~_mnij of Eq. def_Y_oo, V~_mnij)."""
    km, I = P.km, P.I
    N, o = P.nk, P.o
    Vt = np.zeros((N, N, N, o, o, o, o), np.complex128)
    for kmm in km:
        for kn in km:
            for ki in km:
                kj = km.k4(kmm, kn, ki)
                Vt[kmm, kn, ki] = ein("jc,mnic->mnij", t1[kj], I.get("ooov", kmm, kn, ki))
    Y = np.zeros_like(Vt)
    for kmm in km:
        for kn in km:
            for ki in km:
                kj = km.k4(kmm, kn, ki)
                y = Vt[kmm, kn, ki] - Vt[kmm, kn, kj].transpose(0, 1, 3, 2)
                y += I.get("oooo", kmm, kn, ki)
                y += ein("ic,jd,mncd->mnij", t1[ki], t1[kj], I.get("oovv", kmm, kn, ki))
                Y[kmm, kn, ki] = 0.5 * y
    G = np.zeros_like(t2)
    out = np.zeros_like(t2)
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                x = np.zeros(t2.shape[3:], np.complex128)
                for kmm in km:
                    kn = km.k4(ki, kj, kmm)
                    x += ein("mnab,mnij->ijab", t2[kmm, kn, ka], Y[kmm, kn, ki])
                fj = Foo[kj] + 0.5 * ein("jc,nc->nj", t1[kj], Fov[kj])
                fi = Foo[ki] + 0.5 * ein("ic,nc->ni", t1[ki], Fov[ki])
                # - P(ij) sum_n t_{i n}^{ab} (F~_nj + 1/2 t_j^c F~_n^c)   (n carries kj)
                x -= ein("inab,nj->ijab", t2[ki, kj, ka], fj)
                x += ein("jnab,ni->ijab", t2[kj, ki, ka], fi)
                eta = ein("ic,jd->ijcd", t1[ki], t1[kj])
                x -= ein("ijcd,bacd->ijab", eta, I.get("vvvv", kb, ka, ki))
                g = ein("ijcd,racd->rija", eta, I.get("ovvv", kb, ka, ki))
                g += np.conj(I.get("ooov", ki, kj, kb)).transpose(2, 0, 1, 3)
                G[ki, kj, ka] = ein("rb,rija->ijab", t1[kb], g)
                out[ki, kj, ka] = x
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                out[ki, kj, ka] += G[ki, kj, ka] - G[ki, kj, kb].transpose(0, 1, 3, 2)
    return out


def residual(P, t1, t2):
    """(R1, R2) of form B; R2 = A-bar + A-check + A-tilde + A-hat   (Eq. EqDouble)."""
    Foo, Fvv, Fov = fock_tilde(P, t1, t2)
    R1 = residual_t1(P, t1, t2, Foo, Fvv, Fov)
    R2 = a_bar(P, t1, t2) + a_check(P, t1, t2, Fvv, Fov) + a_tilde(P, t1, t2) \
        + a_hat(P, t1, t2, Foo, Fov)
    return R1, R2
