"""Selected rows of the satellite block of S = M X at full size (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For workloads too large for ``adc.sigma_ref`` (the 4-external integrals of
v = 200 alone are 25 GB), the satellite rows are computed one at a time from
their definition: every integral a row needs is assembled from the Cholesky
vectors (Eq. 43) for that row only, and every amplitude from its definition
t_ij^ab = <ab||ij>/D_ij^ab. The terms are those of ``adc.sigma_ref`` (EA:
coupling, zeroth-order diagonal, ladder, ring; IP likewise), Sec. 2.1.

EE doubles rows evaluate the oracle's own term tables (``adc_ee.TERMS``:
the coupling M_SD at first and second order, the second-order overlap and
M_DD^(1)) with the row's four indices held fixed, so that every operand is
a slice assembled from B for that row (and the second-order singles only at
the elements the row needs).
"""
from __future__ import annotations

import numpy as np

__all__ = ["ea_satellite_rows", "ip_satellite_rows", "ee_doubles_rows", "main_rows_ground", "ea_main_rows",
           "ip_main_rows"]


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


# ---------------------------------------------------------------- EE doubles rows

def _class_sel(ch, fixed, o, v, occ):
    base, n = (0, o) if ch in occ else (o, v)
    return base + fixed[ch] if ch in fixed else slice(base, base + n)


def _free(labels, fixed):
    return "".join(ch for ch in labels if ch not in fixed)


class _FixedIndexTensors:
    """The tensors of the EE term tables with some labels held at fixed indices
    (index within the label's class): each array has one axis per free label,
    in label order, and is assembled from B for that slice only."""

    def __init__(self, B, eps_occ, eps_vir, fixed):
        from .adc_ee import _OCC
        self.B = B
        self.eo = np.asarray(eps_occ, np.float64)
        self.ev = np.asarray(eps_vir, np.float64)
        self.o, self.v = self.eo.size, self.ev.size
        self.fixed = dict(fixed)
        self.occ = _OCC
        self._cache = {}
        self._s2 = {}

    def _eri(self, labels):
        """<pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr) (Eq. 43) on the slice."""
        key = ("v", labels, tuple(self.fixed.get(c) for c in labels))
        if key in self._cache:
            return self._cache[key]
        p, q, r, s_ = labels
        sel = lambda c: _class_sel(c, self.fixed, self.o, self.v, self.occ)
        f = lambda *cs: "".join(c for c in cs if c not in self.fixed)
        out = f(p, q, r, s_)
        B = self.B
        val = (np.einsum(f"Q{f(p, r)},Q{f(q, s_)}->{out}", B[:, sel(p), sel(r)], B[:, sel(q), sel(s_)],
                         optimize="greedy")
               - np.einsum(f"Q{f(p, s_)},Q{f(q, r)}->{out}", B[:, sel(p), sel(s_)], B[:, sel(q), sel(r)],
                           optimize="greedy"))
        self._cache[key] = val
        return val

    def _energy(self, ch):
        e = self.eo if ch in self.occ else self.ev
        return e[self.fixed[ch]] if ch in self.fixed else e

    def _denominator(self, a, b, i, j):
        """eps_i + eps_j - eps_a - eps_b on the free labels of (a, b, i, j)."""
        free = _free(a + b + i + j, self.fixed)
        D = np.zeros([self.o if c in self.occ else self.v for c in free]) if free else np.zeros(())
        for ch, sgn in ((a, -1.0), (b, -1.0), (i, 1.0), (j, 1.0)):
            e = self._energy(ch)
            if ch in self.fixed:
                D = D + sgn * e
            else:
                shape = [1] * len(free)
                shape[free.index(ch)] = e.size
                D = D + sgn * e.reshape(shape)
        return D

    def _s2_element(self, a, i):
        """t2_i^a (eps_i - eps_a) = 1/2 sum_jcd <aj||cd> t_ij^cd - 1/2 sum_jkc <jk||ic> t_jk^ac, one element."""
        if (a, i) in self._s2:
            return self._s2[(a, i)]
        sub = _FixedIndexTensors(self.B, self.eo, self.ev, {"a": a, "i": i})
        t_i = sub.array("t1", "cdij")      # t_ij^cd, free c, d, j
        v_a = sub.array("v", "ajcd")       # <aj||cd>, free j, c, d
        t_a = sub.array("t1", "acjk")      # t_jk^ac, free c, j, k
        v_i = sub.array("v", "jkic")       # <jk||ic>, free j, k, c
        num = 0.5 * np.einsum("cdj,jcd->", t_i, v_a) - 0.5 * np.einsum("cjk,jkc->", t_a, v_i)
        val = num / (self.eo[i] - self.ev[a])
        self._s2[(a, i)] = val
        return val

    def array(self, name, labels):
        fx = self.fixed
        if name == "d":
            x, y = labels
            n = self.o if x in self.occ else self.v
            if x in fx and y in fx:
                return np.asarray(1.0 if fx[x] == fx[y] else 0.0)
            if x in fx or y in fx:
                e = np.zeros(n)
                e[fx[x] if x in fx else fx[y]] = 1.0
                return e
            return np.eye(n)
        if name == "v":
            return self._eri(labels)
        if name in ("t1", "t1c"):
            a, b, i, j = labels          # t_ij^ab = <ab||ij> / D_ij^ab
            t = self._eri(a + b + i + j) / self._denominator(a, b, i, j)
            return t.conj() if name == "t1c" else t
        if name in ("s2", "s2c"):
            a, i = labels
            free = _free(labels, fx)
            shape = [self.v if a not in fx else None, self.o if i not in fx else None]
            if not free:
                val = self._s2_element(fx[a], fx[i])
                return np.asarray(np.conj(val) if name == "s2c" else val)
            arr = np.zeros([n for n in shape if n is not None], np.complex128)
            for idx in np.ndindex(*arr.shape):
                it = iter(idx)
                aa = fx[a] if a in fx else next(it)
                ii = fx[i] if i in fx else next(it)
                arr[idx] = self._s2_element(aa, ii)
            return arr.conj() if name == "s2c" else arr
        raise KeyError(name)

    def evaluate(self, key, out):
        """sum over TERMS[key] of coef * product, on the free labels of ``out``."""
        from .adc_ee import TERMS, _TOK
        fout = _free(out, self.fixed)
        total = 0.0
        for coef, product in TERMS[key]:
            subs, ops = [], []
            for name, labs in _TOK.findall(product):
                lab = labs.replace(",", "")
                subs.append(_free(lab, self.fixed))
                ops.append(self.array(name, lab))
            c = float(eval(coef, {"__builtins__": {}}))
            total = total + c * np.einsum(",".join(subs) + "->" + fout, *ops, optimize="greedy")
        return total


def ee_doubles_rows(B, eps_occ, eps_vir, order, x, X, rows, dd_order=1):
    """S2 entries (k<l, c<d) of S = M X for each ``(k, l, c, d)`` in ``rows`` (EE).

    S2_D = sum_S conj(M_SD[S, D]) X1_S + Delta_D X2_D + x [dd_order] sum_D' M_DD^(1)[D, D'] X2_D',
    M_SD = M_SD^(1) + x [(Delta_D - Delta_S) O2 + Z1]  (the blocks of ``adc_ee.Blocks``),
    Delta_S = eps_a - eps_i, Delta_D = eps_c + eps_d - eps_k - eps_l.
    Returns [len(X), len(rows)] complex.
    """
    eo = np.asarray(eps_occ, np.float64)
    ev = np.asarray(eps_vir, np.float64)
    o, v = eo.size, ev.size
    if order == 2:
        x = 0.0
    n1 = o * v
    X = np.atleast_2d(np.asarray(X, np.complex128))
    X1 = X[:, :n1].reshape(-1, o, v)
    X2 = X[:, n1:]
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    pv = av.size
    dS = ev[None, :] - eo[:, None]
    out = np.zeros((X.shape[0], len(rows)), np.complex128)
    for r, (k, l, c, d) in enumerate(rows):
        assert k < l and c < d
        T = _FixedIndexTensors(B, eo, ev, {"k": k, "l": l, "c": c, "d": d})
        Msd = T.evaluate("SD_M1", "iaklcd")
        if x != 0.0:
            dK = ev[c] + ev[d] - eo[k] - eo[l]
            Msd = Msd + x * ((dK - dS) * T.evaluate("SD_O2", "iaklcd") + T.evaluate("SD_Z1", "iaklcd"))
        D = _pair(k, l, o) * pv + _pair(c, d, v)
        val = np.einsum("ia,zia->z", Msd.conj(), X1) + (ev[c] + ev[d] - eo[k] - eo[l]) * X2[:, D]
        if x != 0.0 and dd_order == 1:
            Td = _FixedIndexTensors(B, eo, ev, {"i": k, "j": l, "a": c, "b": d})
            R = Td.evaluate("DD_M1", "ijabklcd")  # [k][l][c][d] free
            Rp = R[io[:, None], jo[:, None], av[None, :], bv[None, :]].reshape(-1)
            val = val + x * (X2 @ Rp)
        out[:, r] = val
    return out



# ---------------------------------------------------------------- IP/EA main rows

def _eri_fixed(B, nocc, spec, fix=None):
    """<pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr) (Eq. 43) for the classes of
    ``spec`` (four of 'o'/'v'), with the positions in ``fix`` held at one
    index (within their class); one axis per free position, in order."""
    fix = fix or {}
    nmo = B.shape[1]
    sel = []
    for pos, c in enumerate(spec):
        base, n = (0, nocc) if c == "o" else (nocc, nmo - nocc)
        sel.append(base + fix[pos] if pos in fix else slice(base, base + n))
    L = "pqrs"

    def lab(*ps):
        return "".join(L[p] for p in ps if p not in fix)

    out = lab(0, 1, 2, 3)
    t1 = np.einsum(f"Q{lab(0, 2)},Q{lab(1, 3)}->{out}", B[:, sel[0], sel[2]], B[:, sel[1], sel[3]],
                   optimize="greedy")
    t2 = np.einsum(f"Q{lab(0, 3)},Q{lab(1, 2)}->{out}", B[:, sel[0], sel[3]], B[:, sel[1], sel[2]],
                   optimize="greedy")
    return t1 - t2


def main_rows_ground(B, eps_occ, eps_vir):
    """Ground-state quantities of ``integrals.Amplitudes`` (first-order doubles
    t1, second-order singles t2s and doubles t2d, the densities gvv and hoo)
    plus the stored integral classes oovv and ovvo, at sizes where the dense
    four-virtual block does not fit: the second-order ladder
    1/2 sum_cd <ab||cd> t_ij^cd is accumulated one virtual index a at a time,
    with <ab||cd> (b > a) for that a assembled from B (Eq. 43); the vovv
    integrals of the second-order singles likewise."""
    eo = np.asarray(eps_occ, np.float64)
    ev = np.asarray(eps_vir, np.float64)
    o, v = eo.size, ev.size
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    g = {"eo": eo, "ev": ev, "o": o, "v": v}
    t1 = _eri_fixed(B, o, "vvoo").transpose(2, 3, 0, 1) / D2        # t_ij^ab = <ab||ij> / D_ij^ab
    tc = t1.conj()
    g["t1"] = t1
    g["oovv"] = _eri_fixed(B, o, "oovv")                               # <ij||ab>
    g["ovvo"] = _eri_fixed(B, o, "ovvo")                               # <kb||cj>
    g["gvv"] = 0.5 * np.einsum("ijdf,ijef->de", tc, t1, optimize="greedy")
    g["hoo"] = 0.5 * np.einsum("njef,mjef->nm", tc, t1, optimize="greedy")
    # second-order singles: (eps_i - eps_a) t_i^a = 1/2 sum_jcd <aj||cd> t_ij^cd - 1/2 sum_jkc <jk||ic> t_jk^ac
    num = -0.5 * np.einsum("jkic,jkac->ia", _eri_fixed(B, o, "ooov"), t1, optimize="greedy")
    Bvv, Bov = B[:, o:, o:], B[:, :o, o:]
    for a in range(v):
        # <aj||cd> = sum_Q (B_ac B_jd - B_ad B_jc): the second product is the first with c, d swapped
        h = np.einsum("Qc,Qjd->jcd", Bvv[:, a, :], Bov, optimize="greedy")
        num[:, a] += 0.5 * np.einsum("jcd,ijcd->i", h - h.transpose(0, 2, 1), t1, optimize="greedy")
    g["t2s"] = num / (eo[:, None] - ev[None, :])
    # second-order doubles: D t2 = 1/2 <ab||cd> t^cd + 1/2 <kl||ij> t_kl + P(ij) P(ab) sum_kc <kb||cj> t_ik^ac
    ring = np.einsum("kbcj,ikac->ijab", g["ovvo"], t1, optimize="greedy")
    t2 = ring - ring.transpose(1, 0, 2, 3) - ring.transpose(0, 1, 3, 2) + ring.transpose(1, 0, 3, 2)
    del ring
    t2 += 0.5 * np.einsum("klij,klab->ijab", _eri_fixed(B, o, "oooo"), t1, optimize="greedy")
    # ladder 1/2 sum_cd <ab||cd> t_ij^cd = sum_{c<d} <ab||cd> t_ij^cd (both antisymmetric in c, d),
    # for b > a from <ab||cd> = sum_Q (B_ac B_bd - B_ad B_bc); b < a by its antisymmetry in a, b
    iu, ju = np.triu_indices(v, 1)
    t1p = t1[:, :, iu, ju]
    lad = np.zeros_like(t1)
    for a in range(v - 1):
        h = np.einsum("Qc,Qbd->bcd", Bvv[:, a, :], Bvv[:, a + 1:, :], optimize="greedy")
        G = h - h.transpose(0, 2, 1)
        lad[:, :, a, a + 1:] = np.einsum("bp,ijp->ijb", G[:, iu, ju], t1p, optimize="greedy")
    lad -= lad.transpose(0, 1, 3, 2)
    g["t2d"] = (t2 + lad) / D2
    return g


def ea_main_rows(B, eps_occ, eps_vir, order, x, X, rows, ground=None):
    """S1 entries (the 1p rows) c of S = M X for each c in ``rows`` (EA).

    S1_c = sum_b M11_cb X1_b + 1/2 sum_kde (<ck||de> + x M12^(2)_c,kde) X2_kde,
    M11 = M0 + M2 (+ x M3 at order 3), term by term as ``adc.main_block`` writes
    them, with every integral the row needs assembled from B for that row
    (Eq. 43). The four-virtual term 1/4 sum <cd||be> conj(t_ij^cd) t_ij^ea is
    contracted through B: sum_cde <cd||be> P_cde = sum_Q [sum_c B_cb sum_de B_de
    P_cde - sum_d B_db sum_ce B_ce P_cde]. Returns [len(X), len(rows)] complex.
    """
    g = ground if ground is not None else main_rows_ground(B, eps_occ, eps_vir)
    eo, ev, o, v = g["eo"], g["ev"], g["o"], g["v"]
    if order == 2:
        x = 0.0
    t1, t2d, t2s, gvv, hoo = g["t1"], g["t2d"], g["t2s"], g["gvv"], g["hoo"]
    tc = t1.conj()
    X = np.atleast_2d(np.asarray(X, np.complex128))
    X1 = X[:, :v]
    iu, ju = np.triu_indices(v, 1)
    X2f = np.zeros((X.shape[0], o, v, v), np.complex128)
    X2f[:, :, iu, ju] = X[:, v:].reshape(X.shape[0], o, iu.size)
    X2f[:, :, ju, iu] = -X2f[:, :, iu, ju]
    Bvv = B[:, o:, o:]
    out = np.zeros((X.shape[0], len(rows)), np.complex128)
    for r, a in enumerate(rows):
        de = ev[a] - ev                                           # eps_a - eps_b
        m11 = np.zeros(v, np.complex128)
        m11[a] = ev[a]
        m11 += -0.5 * np.einsum("klc,klbc->b", t1[:, :, a, :], g["oovv"], optimize="greedy") + 0.5 * de * gvv[:, a]
        if x != 0.0:
            g3 = 0.5 * (np.einsum("ijbf,ijf->b", tc, t2d[:, :, a, :], optimize="greedy")
                        + np.einsum("ijbf,ijf->b", t2d.conj(), t1[:, :, a, :], optimize="greedy"))
            P = np.einsum("ijcd,ije->cde", tc, t1[:, :, :, a], optimize="greedy")      # P_cde for e a-paired
            U = np.einsum("Qde,cde->Qc", Bvv, P, optimize="greedy")
            W = np.einsum("Qce,cde->Qd", Bvv, P, optimize="greedy")
            four = np.einsum("Qcb,Qc->b", Bvv, U, optimize="greedy") - np.einsum("Qdb,Qd->b", Bvv, W,
                                                                                optimize="greedy")
            R = np.einsum("njcf,mjf->cnm", tc, t1[:, :, a, :], optimize="greedy")       # R_ca,nm
            y3 = (-0.5 * np.einsum("klc,klbc->b", t2d[:, :, a, :], g["oovv"], optimize="greedy")
                  - np.einsum("mbd,md->b", _eri_fixed(B, o, "ovvv", {1: a}), t2s, optimize="greedy")
                  + np.einsum("dbk,kd->b", _eri_fixed(B, o, "vvvo", {0: a}), t2s.conj(), optimize="greedy")
                  + np.einsum("dbe,de->b", _eri_fixed(B, o, "vvvv", {0: a}), gvv, optimize="greedy")
                  + 0.25 * four
                  + np.einsum("mbn,nm->b", _eri_fixed(B, o, "ovvo", {1: a}), hoo, optimize="greedy")
                  - np.einsum("mcbn,cnm->b", g["ovvo"], R, optimize="greedy"))
            m11 += x * (y3 + 0.5 * de * g3)
        C = _eri_fixed(B, o, "vovv", {0: a})                                     # <ak||de>
        if x != 0.0:
            c2 = (0.5 * np.einsum("kmn,mnde->kde", _eri_fixed(B, o, "vooo", {0: a}), tc, optimize="greedy")
                  + np.einsum("gem,kmgd->kde", _eri_fixed(B, o, "vvvo", {0: a}), tc, optimize="greedy")
                  - np.einsum("gdm,kmge->kde", _eri_fixed(B, o, "vvvo", {0: a}), tc, optimize="greedy"))
            C = C + x * c2
        out[:, r] = X1 @ m11 + 0.5 * np.einsum("kde,zkde->z", C, X2f, optimize="greedy")
    return out


def ip_main_rows(B, eps_occ, eps_vir, order, x, X, rows, ground=None):
    """S1 entries (the 1h rows) k of S = M X for each k in ``rows`` (IP).

    S1_k = sum_l M11_kl X1_l + 1/2 sum_ija (<ji||ak> + x M12^(2)_k,ija) X2_ija,
    M11 = M0 + M2 (+ x M3 at order 3), term by term as ``adc.main_block``
    writes them, every integral of the row assembled from B (Eq. 43).
    Returns [len(X), len(rows)] complex.
    """
    g = ground if ground is not None else main_rows_ground(B, eps_occ, eps_vir)
    eo, ev, o, v = g["eo"], g["ev"], g["o"], g["v"]
    if order == 2:
        x = 0.0
    t1, t2d, t2s, gvv, hoo = g["t1"], g["t2d"], g["t2s"], g["gvv"], g["hoo"]
    tc = t1.conj()
    X = np.atleast_2d(np.asarray(X, np.complex128))
    X1 = X[:, :o]
    iu, ju = np.triu_indices(o, 1)
    X2f = np.zeros((X.shape[0], o, o, v), np.complex128)
    X2f[:, iu, ju, :] = X[:, o:].reshape(X.shape[0], iu.size, v)
    X2f[:, ju, iu, :] = -X2f[:, iu, ju, :]
    out = np.zeros((X.shape[0], len(rows)), np.complex128)
    vovo = _eri_fixed(B, o, "vovo") if x != 0.0 else None          # <cj||dk>
    for r, i in enumerate(rows):
        do = eo[i] - eo                                             # eps_i - eps_j
        m11 = np.zeros(o, np.complex128)
        m11[i] = -eo[i]
        m11 += 0.5 * np.einsum("kjcd,kcd->j", g["oovv"], t1[i], optimize="greedy") - 0.5 * do * hoo[:, i]
        if x != 0.0:
            h3 = 0.5 * (np.einsum("jkcd,kcd->j", tc, t2d[i], optimize="greedy")
                        + np.einsum("jkcd,kcd->j", t2d.conj(), t1[i], optimize="greedy"))
            Pk = np.einsum("lmef,kef->lmk", tc, t1[i], optimize="greedy")
            Z = np.einsum("klcf,ldf->ckd", tc, t1[i], optimize="greedy")
            y3 = (0.5 * np.einsum("kjcd,kcd->j", g["oovv"], t2d[i], optimize="greedy")
                  - np.einsum("kje,ke->j", _eri_fixed(B, o, "oovo", {3: i}), t2s, optimize="greedy")
                  + np.einsum("cjk,kc->j", _eri_fixed(B, o, "vooo", {2: i}), t2s.conj(), optimize="greedy")
                  + np.einsum("kjl,lk->j", _eri_fixed(B, o, "oooo", {3: i}), hoo, optimize="greedy")
                  + 0.25 * np.einsum("kjlm,lmk->j", _eri_fixed(B, o, "oooo"), Pk, optimize="greedy")
                  - np.einsum("cjd,cd->j", _eri_fixed(B, o, "vovo", {3: i}), gvv, optimize="greedy")
                  + np.einsum("cjdk,ckd->j", vovo, Z, optimize="greedy"))
            m11 += x * (y3 - 0.5 * do * h3)
        C = _eri_fixed(B, o, "oovo", {3: i}).transpose(1, 0, 2)              # <ji||ak> -> [i][j][a]
        if x != 0.0:
            c2 = (0.5 * np.einsum("efa,jief->ija", _eri_fixed(B, o, "vvvo", {3: i}), tc, optimize="greedy")
                  - np.einsum("fim,jmfa->ija", _eri_fixed(B, o, "vooo", {3: i}), tc, optimize="greedy")
                  + np.einsum("fjm,imfa->ija", _eri_fixed(B, o, "vooo", {3: i}), tc, optimize="greedy"))
            C = C + x * c2
        out[:, r] = X1 @ m11 + 0.5 * np.einsum("ija,zija->z", C, X2f, optimize="greedy")
    return out
