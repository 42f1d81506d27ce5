"""Selected rows of the satellite block of S = M X at full size (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For workloads too large for ``adc.sigma_ref`` (the 4-external integrals of
v = 200 alone are 25 GB), the satellite rows are computed one at a time from
their definition: every integral a row needs is assembled from the Cholesky
vectors (Eq. 43) for that row only, and every amplitude from its definition
t_ij^ab = <ab||ij>/D_ij^ab. The terms are those of ``adc.sigma_ref`` (EA:
coupling, zeroth-order diagonal, ladder, ring; IP likewise), Sec. 2.1.
"""
from __future__ import annotations

import numpy as np

__all__ = ["ea_satellite_rows", "ip_satellite_rows"]


def _pair(p, q, n):
    return p * n - p * (p + 1) // 2 + (q - p - 1)


def _ea_full(X2row_k, v):
    """Packed [npairs_v] -> antisymmetric [v][v] for one occupied index."""
    iu, ju = np.triu_indices(v, 1)
    F = np.zeros((v, v), np.complex128)
    F[iu, ju] = X2row_k
    F[ju, iu] = -X2row_k
    return F


def ea_satellite_rows(B, eps_occ, eps_vir, order, x, X, rows):
    """S2 entries (k, d<e) for each ``(k, d, e)`` in ``rows`` and each vector in X.

    S2_kde = sum_c conj(C_c,kde) X1_c + (eps_d + eps_e - eps_k) X2_kde
             + x [ sum_{f<g} <de||fg> X2_kfg - sum_lf (<dl||fk> X2f_lfe - <el||fk> X2f_lfd) ]
    C_c,kde = <ck||de> + x [1/2 sum_mn <ck||mn> conj(t_mn^de)
                            + sum_gm (<cg||em> conj(t_km^gd) - <cg||dm> conj(t_km^ge))]
    Returns [len(X), len(rows)] complex.
    """
    eo = np.asarray(eps_occ, np.float64)
    ev = np.asarray(eps_vir, np.float64)
    o, v = eo.size, ev.size
    if order == 2:
        x = 0.0
    pv = v * (v - 1) // 2
    X = np.atleast_2d(X)
    X1 = X[:, :v]
    X2 = X[:, v:].reshape(X.shape[0], o, pv)
    O, V = slice(0, o), slice(o, o + v)
    Bvv, Bvo, Bov, Boo = B[:, V, V], B[:, V, O], B[:, O, V], B[:, O, O]
    out = np.zeros((X.shape[0], len(rows)), np.complex128)
    for r, (k, d, e) in enumerate(rows):
        assert d < e
        # <ck||de> for all c
        ck_de = np.einsum("Qc,Q->c", Bvv[:, :, d], Bov[:, k, e]) - np.einsum("Qc,Q->c", Bvv[:, :, e], Bov[:, k, d])
        C = ck_de
        if x != 0.0:
            # t_mn^de for all m, n
            de_mn = (np.einsum("Qm,Qn->mn", Bvo[:, d, :], Bvo[:, e, :])
                     - np.einsum("Qn,Qm->mn", Bvo[:, d, :], Bvo[:, e, :]))
            Dmn = eo[:, None] + eo[None, :] - ev[d] - ev[e]
            t_de = de_mn / Dmn
            # <ck||mn> for all c, m, n
            ck_mn = (np.einsum("Qcm,Qn->cmn", Bvo, Boo[:, k, :]) - np.einsum("Qcn,Qm->cmn", Bvo, Boo[:, k, :]))
            termA = 0.5 * np.einsum("cmn,mn->c", ck_mn, t_de.conj())
            # t_km^gd and t_km^ge for all g, m
            def t_k_xd(dd):
                num = (np.einsum("Qg,Qm->gm", Bvo[:, :, k], Bvo[:, dd, :])
                       - np.einsum("Qgm,Q->gm", Bvo, Bvo[:, dd, k]))  # <g dd||k m>
                den = eo[k] + eo[None, :] - ev[:, None] - ev[dd]
                return num / den  # [g, m] = t_km^{g dd}
            tgd = t_k_xd(d)
            tge = t_k_xd(e)
            # <cg||em> for all c, g, m = sum_Q (B_ce B_gm - B_cm B_ge)
            def cg_xm(xx):
                return (np.einsum("Qc,Qgm->cgm", Bvv[:, :, xx], Bvo)
                        - np.einsum("Qcm,Qg->cgm", Bvo, Bvv[:, :, xx]))
            termB = (np.einsum("cgm,gm->c", cg_xm(e), tgd.conj()) - np.einsum("cgm,gm->c", cg_xm(d), tge.conj()))
            C = ck_de + x * (termA + termB)
        val = X1 @ C.conj()
        val = val + (ev[d] + ev[e] - eo[k]) * X2[:, k, _pair(d, e, v)]
        if x != 0.0:
            # ladder: <de||fg> for f < g
            de_fg = (np.einsum("Qf,Qg->fg", Bvv[:, d, :], Bvv[:, e, :])
                     - np.einsum("Qg,Qf->fg", Bvv[:, d, :], Bvv[:, e, :]))
            iu, ju = np.triu_indices(v, 1)
            lad = X2[:, k, :] @ de_fg[iu, ju]
            # ring: sum_lf <dl||fk> X2f_lfe - <el||fk> X2f_lfd, <dl||fk> = sum_Q (B_df B_lk - B_dk B_lf)
            def ring(dd, ee):
                W = (np.einsum("Qf,Ql->lf", Bvv[:, dd, :], Boo[:, :, k])
                     - np.einsum("Q,Qlf->lf", Bvo[:, dd, k], Bov))
                acc = np.zeros(X.shape[0], np.complex128)
                for l in range(o):
                    for vec in range(X.shape[0]):
                        F = _ea_full(X2[vec, l, :], v)
                        acc[vec] += W[l] @ F[:, ee]
                return acc
            val = val + x * (lad - (ring(d, e) - ring(e, d)))
        out[:, r] = val
    return out


def ip_satellite_rows(B, eps_occ, eps_vir, order, x, X, rows):
    """S2 entries (i<j, a) for each ``(i, j, a)`` in ``rows``.

    S2_ija = sum_k conj(C_k,ija) X1_k + (eps_a - eps_i - eps_j) X2_ija
             + x [ sum_{k<l} <kl||ij> X2_kla + sum_kb (<ak||bj> X2f_kib - <ak||bi> X2f_kjb) ]
    C_k,ija = <ji||ak> + x [1/2 sum_ef <ef||ak> conj(t_ji^ef)
                            - sum_fm <fi||mk> conj(t_jm^fa) + sum_fm <fj||mk> conj(t_im^fa)]
    """
    eo = np.asarray(eps_occ, np.float64)
    ev = np.asarray(eps_vir, np.float64)
    o, v = eo.size, ev.size
    if order == 2:
        x = 0.0
    po = o * (o - 1) // 2
    X = np.atleast_2d(X)
    X1 = X[:, :o]
    X2 = X[:, o:].reshape(X.shape[0], po, v)
    O, V = slice(0, o), slice(o, o + v)
    Bvv, Bvo, Bov, Boo = B[:, V, V], B[:, V, O], B[:, O, V], B[:, O, O]

    def X2f(vec, p, q, a):
        if p == q:
            return 0.0
        if p < q:
            return X2[vec, _pair(p, q, o), a]
        return -X2[vec, _pair(q, p, o), a]

    out = np.zeros((X.shape[0], len(rows)), np.complex128)
    for r, (i, j, a) in enumerate(rows):
        assert i < j
        # <ji||ak> for all k = sum_Q (B_ja B_ik - B_jk B_ia)
        C = np.einsum("Q,Qk->k", Bov[:, j, a], Boo[:, i, :]) - np.einsum("Qk,Q->k", Boo[:, j, :], Bov[:, i, a])
        if x != 0.0:
            # t_ji^ef for all e, f
            ef_ji = (np.einsum("Qe,Qf->ef", Bvo[:, :, j], Bvo[:, :, i])
                     - np.einsum("Qe,Qf->ef", Bvo[:, :, i], Bvo[:, :, j]))
            Def = eo[j] + eo[i] - ev[:, None] - ev[None, :]
            t_ji = ef_ji / Def
            # <ef||ak> for all e, f, k = sum_Q (B_ea B_fk - B_ek B_fa)
            ef_ak = (np.einsum("Qe,Qfk->efk", Bvv[:, :, a], Bvo) - np.einsum("Qek,Qf->efk", Bvo, Bvv[:, :, a]))
            termA = 0.5 * np.einsum("efk,ef->k", ef_ak, t_ji.conj())

            def t_x_m_fa(ii):
                # t_{ii m}^{f a} for all m, f
                num = (np.einsum("Qf,Qm->mf", Bvo[:, :, ii], Bvo[:, a, :])
                       - np.einsum("Qfm,Q->mf", Bvo, Bvo[:, a, ii]))
                den = eo[ii] + eo[:, None] - ev[None, :] - ev[a]
                return num / den
            tj = t_x_m_fa(j)
            ti = t_x_m_fa(i)

            def f_x_mk(ii):
                # <f ii||m k> for all f, m, k = sum_Q (B_fm B_ik - B_fk B_im)
                return (np.einsum("Qfm,Qk->fmk", Bvo, Boo[:, ii, :]) - np.einsum("Qfk,Qm->fmk", Bvo, Boo[:, ii, :]))
            termB = -np.einsum("fmk,mf->k", f_x_mk(i), tj.conj()) + np.einsum("fmk,mf->k", f_x_mk(j), ti.conj())
            C = C + x * (termA + termB)
        val = X1 @ C.conj()
        val = val + (ev[a] - eo[i] - eo[j]) * X2[:, _pair(i, j, o), a]
        if x != 0.0:
            # ladder: <kl||ij> for k < l
            kl_ij = (np.einsum("Qk,Ql->kl", Boo[:, :, i], Boo[:, :, j]) - np.einsum("Qk,Ql->kl", Boo[:, :, j], Boo[:, :, i]))
            iu, ju = np.triu_indices(o, 1)
            lad = X2[:, :, a] @ kl_ij[iu, ju]

            def ring(ii, jj):
                # sum_kb <ak||b jj> X2f_{k ii b}, <ak||bj> = sum_Q (B_ab B_kj - B_aj B_kb)
                W = (np.einsum("Qb,Qk->kb", Bvv[:, a, :], Boo[:, :, jj]) - np.einsum("Q,Qkb->kb", Bvo[:, a, jj], Bov))
                acc = np.zeros(X.shape[0], np.complex128)
                for vec in range(X.shape[0]):
                    for k in range(o):
                        for b in range(v):
                            acc[vec] += W[k, b] * X2f(vec, k, ii, b)
                return acc
            val = val + x * (lad + ring(i, j) - ring(j, i))
        out[:, r] = val
    return out
