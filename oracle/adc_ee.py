"""Closed-form EE-ADC(2), ADC(2)+x(3), ADC(3) blocks and sigma product (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Excitation manifold (Sec. 2.1, Eq. 2): singles ``a+_a a_i |Psi0>`` and
doubles ``a+_a a_i a+_b a_j |Psi0> = a+_a a+_b a_j a_i |Psi0>`` (i<j, a<b).
The singles precursors are Gram-Schmidt orthogonalised against the ground
state (Eq. 5), so with ``E_bj = a+_b a_j`` and the normalised MP ground state

    S_ia,jb = <E_ai^+ E_bj> - <E_ai^+><E_bj>,   K_ia,jb = <E_ai^+ [H, E_bj]>,
    M_SS = S^-1/2 K S^-1/2                                    (Eqs. 6-7).

Expanding with H - E0 = F_N + V_N and [F_N, E_bj] = (eps_b - eps_j) E_bj:

    M_SS^(1) = K1,   M_SS^(2) = W o S2 + Y2,
    M_SS^(3) = W o S3 + Y3 - 1/2 (S2 K1 + K1 S2),   W_ia,jb = ((eps_b-eps_j) - (eps_a-eps_i))/2,

where S2, S3 are the connected parts of <E_ai^+ E_bj> at second and third
order and Y = <E_ai^+ [V_N, E_bj]> (Y2 from Psi1, Y3 from Psi1 x Psi1 and
Psi2). The coupling to the doubles class (precursors orthogonalised against
Psi0 and the singles) is, through second order,

    M_SD^(1) = <Phi| E_S^+ [V_N, C_K] |Phi>,
    M_SD^(2) = (Delta_K - Delta_S) <E_S^+ C_K>^(2) + <E_S^+ [V_N, C_K]>^(1),

and the doubles block is diag(eps_a + eps_b - eps_i - eps_j) plus, at third
order, the first-order M_DD^(1) = <Phi_D| V_N |Phi_D'>.

Each expectation value was evaluated with Wick's theorem (first-order
amplitudes t1, second-order doubles t2 and singles s2 of ``integrals``;
``v(pq,rs)`` = <pq||rs> of Eq. 43). The term table below lists the result:
one line per term, a rational coefficient and a product of tensors with
upper,lower index labels, ``t1(ab,ij)`` = t_ij^ab, ``t1c`` its complex
conjugate, ``s2(a,i)`` = t2_i^a, ``d(xy)`` a Kronecker delta. Lower-case
labels are the free indices (i, j, k, l occupied; a, b, c, d virtual),
upper-case labels are summed (M..W occupied, A..H virtual). Every block and
order is pinned element by element against the brute-force ISR series.

As for IP/EA, ADC(2)+x(3) scales every term ADC(3) adds (M_SS^(3), M_SD^(2),
M_DD^(1)) by x; ``dd_order=0`` drops M_DD^(1) alone (the doubles block kept
at the ADC(2) level).
"""
from __future__ import annotations

import re

import numpy as np

from .integrals import Amplitudes, eri

__all__ = ["TERMS", "dims", "Tensors", "Blocks", "explicit_matrix", "sigma_ref", "diagonal_ref",
           "unpack2", "pack2"]

TERMS = {
    "SS_K1": [
        ("-1", "v(aj,bi)"),
    ],
    "SS_S2": [
        ("1", "t1(aA,iM) t1c(bA,jM)"),
        ("-1/2", "t1(aA,MN) t1c(bA,MN) d(ij)"),
        ("-1/2", "t1(AB,iM) t1c(AB,jM) d(ab)"),
        ("1/4", "t1(AB,MN) t1c(AB,MN) d(ab) d(ij)"),
    ],
    "SS_Y2": [
        ("1", "t1(aA,iM) v(jM,bA)"),
        ("-1/2", "t1(aA,MN) v(MN,bA) d(ij)"),
        ("-1/2", "t1(AB,iM) v(jM,AB) d(ab)"),
    ],
    "SS_S3": [
        ("1", "t1(aA,iM) t2c(bA,jM)"),
        ("1", "t1c(bA,jM) t2(aA,iM)"),
        ("-1/2", "t1(aA,MN) t2c(bA,MN) d(ij)"),
        ("-1/2", "t1(AB,iM) t2c(AB,jM) d(ab)"),
        ("-1/2", "t1c(bA,MN) t2(aA,MN) d(ij)"),
        ("-1/2", "t1c(AB,jM) t2(AB,iM) d(ab)"),
        ("1/4", "t1(AB,MN) t2c(AB,MN) d(ab) d(ij)"),
        ("1/4", "t1c(AB,MN) t2(AB,MN) d(ab) d(ij)"),
    ],
    "SS_Y3a": [
        ("1", "t1(aA,iM) t1c(AB,jN) v(BM,bN)"),
        ("1", "t1(aA,iM) t1c(AB,MN) v(jB,bN)"),
        ("1/2", "t1(aA,iM) t1c(bA,NO) v(jM,NO)"),
        ("1/2", "t1(aA,iM) t1c(BC,jM) v(BC,bA)"),
        ("1/2", "t1(aA,MN) t1c(bB,MN) v(jB,iA)"),
        ("1/2", "t1(aA,MN) t1c(AB,MN) v(jB,bi)"),
        ("1/2", "t1(AB,iM) t1c(AB,jN) v(aM,bN)"),
        ("1/2", "t1(AB,MN) t1c(bA,MN) v(aj,iB)"),
        ("-1", "t1(aA,iM) t1c(bB,MN) v(jB,AN)"),
        ("-1", "t1(aA,MN) t1c(bA,MO) v(jN,iO)"),
        ("-1", "t1(aA,MN) t1c(AB,jM) v(BN,bi)"),
        ("-1", "t1(AB,iM) t1c(bA,MN) v(aj,BN)"),
        ("-1", "t1(AB,iM) t1c(AC,jM) v(aC,bB)"),
        ("-1/2", "t1(AB,iM) t1c(AB,MN) v(aj,bN)"),
        ("-1/2", "t1(AB,MN) t1c(AB,jM) v(aN,bi)"),
        ("-1/4", "t1(AB,MN) t1c(AB,MN) v(aj,bi)"),
        ("1", "t1(AB,iM) t1c(AC,MN) v(jC,BN) d(ab)"),
        ("1/2", "t1(AB,MN) t1c(AB,MO) v(jN,iO) d(ab)"),
        ("1/2", "t1(AB,MN) t1c(AC,MN) v(aC,bB) d(ij)"),
        ("-1", "t1(aA,MN) t1c(AB,MO) v(BN,bO) d(ij)"),
        ("-1/2", "t1(AB,MN) t1c(AB,MO) v(aN,bO) d(ij)"),
        ("-1/2", "t1(AB,MN) t1c(AC,MN) v(jC,iB) d(ab)"),
        ("-1/4", "t1(aA,MN) t1c(BC,MN) v(BC,bA) d(ij)"),
        ("-1/4", "t1(AB,iM) t1c(AB,NO) v(jM,NO) d(ab)"),
    ],
    "SS_Y3b": [
        ("1", "t2(aA,iM) v(jM,bA)"),
        ("-1", "s2(a,M) v(jM,bi)"),
        ("-1", "s2(A,i) v(aj,bA)"),
        ("-1", "s2c(b,M) v(aj,iM)"),
        ("-1", "s2c(A,j) v(aA,bi)"),
        ("1", "s2(A,M) v(aM,bA) d(ij)"),
        ("1", "s2c(A,M) v(aA,bM) d(ij)"),
        ("-1", "s2(A,M) v(jM,iA) d(ab)"),
        ("-1", "s2c(A,M) v(jA,iM) d(ab)"),
        ("-1/2", "t2(aA,MN) v(MN,bA) d(ij)"),
        ("-1/2", "t2(AB,iM) v(jM,AB) d(ab)"),
    ],
    "SD_M1": [
        ("1", "v(al,cd) d(ik)"),
        ("1", "v(kl,di) d(ac)"),
        ("-1", "v(ak,cd) d(il)"),
        ("-1", "v(kl,ci) d(ad)"),
    ],
    "SD_O2": [
        ("1", "s2c(c,k) d(ad) d(il)"),
        ("1", "s2c(d,l) d(ac) d(ik)"),
        ("-1", "s2c(c,l) d(ad) d(ik)"),
        ("-1", "s2c(d,k) d(ac) d(il)"),
    ],
    "SD_Z1": [
        ("1", "t1c(cd,lM) v(ak,iM)"),
        ("1", "t1c(dA,kl) v(aA,ci)"),
        ("-1", "t1c(cd,kM) v(al,iM)"),
        ("-1", "t1c(cA,kl) v(aA,di)"),
        ("1", "t1c(cA,kM) v(aA,dM) d(il)"),
        ("1", "t1c(cA,lM) v(kA,iM) d(ad)"),
        ("1", "t1c(dA,kM) v(lA,iM) d(ac)"),
        ("1", "t1c(dA,lM) v(aA,cM) d(ik)"),
        ("1/2", "t1c(cd,MN) v(al,MN) d(ik)"),
        ("1/2", "t1c(AB,kl) v(AB,di) d(ac)"),
        ("-1", "t1c(cA,kM) v(lA,iM) d(ad)"),
        ("-1", "t1c(cA,lM) v(aA,dM) d(ik)"),
        ("-1", "t1c(dA,kM) v(aA,cM) d(il)"),
        ("-1", "t1c(dA,lM) v(kA,iM) d(ac)"),
        ("-1/2", "t1c(cd,MN) v(ak,MN) d(il)"),
        ("-1/2", "t1c(AB,kl) v(AB,ci) d(ad)"),
        ("1/2", "t1c(cA,MN) v(lA,MN) d(ad) d(ik)"),
        ("1/2", "t1c(dA,MN) v(kA,MN) d(ac) d(il)"),
        ("1/2", "t1c(AB,kM) v(AB,cM) d(ad) d(il)"),
        ("1/2", "t1c(AB,lM) v(AB,dM) d(ac) d(ik)"),
        ("-1/2", "t1c(cA,MN) v(kA,MN) d(ad) d(il)"),
        ("-1/2", "t1c(dA,MN) v(lA,MN) d(ac) d(ik)"),
        ("-1/2", "t1c(AB,kM) v(AB,dM) d(ac) d(il)"),
        ("-1/2", "t1c(AB,lM) v(AB,cM) d(ad) d(ik)"),
    ],
    "DD_M1": [
        ("1", "v(ab,cd) d(ik) d(jl)"),
        ("1", "v(ak,cj) d(bd) d(il)"),
        ("1", "v(ak,di) d(bc) d(jl)"),
        ("1", "v(al,ci) d(bd) d(jk)"),
        ("1", "v(al,dj) d(bc) d(ik)"),
        ("1", "v(bk,ci) d(ad) d(jl)"),
        ("1", "v(bk,dj) d(ac) d(il)"),
        ("1", "v(bl,cj) d(ad) d(ik)"),
        ("1", "v(bl,di) d(ac) d(jk)"),
        ("1", "v(kl,ij) d(ac) d(bd)"),
        ("-1", "v(ab,cd) d(il) d(jk)"),
        ("-1", "v(ak,ci) d(bd) d(jl)"),
        ("-1", "v(ak,dj) d(bc) d(il)"),
        ("-1", "v(al,cj) d(bd) d(ik)"),
        ("-1", "v(al,di) d(bc) d(jk)"),
        ("-1", "v(bk,cj) d(ad) d(il)"),
        ("-1", "v(bk,di) d(ac) d(jl)"),
        ("-1", "v(bl,ci) d(ad) d(jk)"),
        ("-1", "v(bl,dj) d(ac) d(ik)"),
        ("-1", "v(kl,ij) d(ad) d(bc)"),
    ],
}

_OCC = set("ijklMNOPRSTW")
_VIR = set("abcdABCDEFGH")
_TOK = re.compile(r"([a-z0-9]+)\(([A-Za-z,]+)\)")


def dims(nocc, nvir):
    return nocc * nvir, (nocc * (nocc - 1) // 2) * (nvir * (nvir - 1) // 2)


class Tensors:
    """Arrays the term table refers to, for one problem."""

    def __init__(self, B, eps_occ, eps_vir, amp=None):
        self.amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir)
        self.B, self.o, self.v = B, self.amp.nocc, self.amp.nvir
        self._eri = {}

    def _type(self, ch):
        return "o" if ch in _OCC else "v"

    def array(self, name, labels):
        """Array with one axis per label, in label order."""
        if name == "d":
            n = self.o if self._type(labels[0]) == "o" else self.v
            return np.eye(n)
        if name == "v":
            spec = "".join(self._type(c) for c in labels)
            if spec not in self._eri:
                self._eri[spec] = eri(self.B, self.o, spec)
            return self._eri[spec]
        a = self.amp
        if name in ("t1", "t1c", "t2", "t2c"):
            t = a.t1 if name.startswith("t1") else a.t2d  # [i, j, a, b]
            t = t.transpose(2, 3, 0, 1)  # labels are (a b, i j)
            return t.conj() if name.endswith("c") else t
        if name in ("s2", "s2c"):
            s = a.t2s.T  # labels are (a, i)
            return s.conj() if name.endswith("c") else s
        raise KeyError(name)

    def term_operands(self, product):
        subs, ops = [], []
        for name, labs in _TOK.findall(product):
            lab = labs.replace(",", "")
            subs.append(lab)
            ops.append(self.array(name, lab))
        return subs, ops

    def evaluate(self, key, out, extra=(), conj=False):
        """sum over the rows of TERMS[key] of coef * product (* extra operands).

        ``extra`` is a list of (labels, array) appended to every product;
        ``conj`` takes the complex conjugate of the table's product (not of extra).
        """
        total = 0.0
        for coef, product in TERMS[key]:
            subs, ops = self.term_operands(product)
            if conj:
                ops = [np.conj(x) for x in ops]
            for lab, arr in extra:
                subs.append(lab)
                ops.append(arr)
            c = float(eval(coef, {"__builtins__": {}}))
            total = total + c * np.einsum(",".join(subs) + "->" + out, *ops, optimize=True)
        return total


def _pairs(n):
    return np.triu_indices(n, 1)


def unpack2(X2, nocc, nvir):
    """[k][npairs_o*npairs_v] -> [k, i, j, a, b] antisymmetric in (i,j) and (a,b)."""
    X2 = np.atleast_2d(X2)
    k = X2.shape[0]
    io, jo = _pairs(nocc)
    av, bv = _pairs(nvir)
    Y = X2.reshape(k, io.size, av.size)
    F = np.zeros((k, nocc, nocc, nvir, nvir), np.complex128)
    for s_o, (p, q) in ((1, (io, jo)), (-1, (jo, io))):
        for s_v, (r, t) in ((1, (av, bv)), (-1, (bv, av))):
            F[:, p[:, None], q[:, None], r[None, :], t[None, :]] = (s_o * s_v) * Y
    return F


def pack2(F, nocc, nvir):
    io, jo = _pairs(nocc)
    av, bv = _pairs(nvir)
    k = F.shape[0]
    return F[:, io[:, None], jo[:, None], av[None, :], bv[None, :]].reshape(k, -1)


class Blocks:
    """Order-resolved dense EE blocks for a small case."""

    def __init__(self, B, eps_occ, eps_vir):
        T = Tensors(B, eps_occ, eps_vir)
        self.T = T
        o, v = T.o, T.v
        eo, ev = T.amp.eo, T.amp.ev
        n1 = o * v
        ev_ = lambda k, out, shape: T.evaluate(k, out).reshape(shape)
        K1 = ev_("SS_K1", "iajb", (n1, n1))
        t = T.amp
        N2 = 0.25 * np.sum(np.abs(t.t1) ** 2)
        N3 = 0.5 * np.real(np.sum(t.t1.conj() * t.t2d))
        I = np.eye(n1)
        S2 = ev_("SS_S2", "iajb", (n1, n1)) - N2 * I
        S3 = ev_("SS_S3", "iajb", (n1, n1)) - N3 * I
        Y2 = ev_("SS_Y2", "iajb", (n1, n1))
        Y3 = ev_("SS_Y3a", "iajb", (n1, n1)) + ev_("SS_Y3b", "iajb", (n1, n1)) - N2 * K1
        dS = (ev[None, :] - eo[:, None]).reshape(-1)
        W = 0.5 * (dS[None, :] - dS[:, None])
        self.MSS = [np.diag(dS).astype(np.complex128), K1, W * S2 + Y2,
                    W * S3 + Y3 - 0.5 * (S2 @ K1 + K1 @ S2)]
        io, jo = _pairs(o)
        av, bv = _pairs(v)
        pk = lambda F: F[:, :, io[:, None], jo[:, None], av[None, :], bv[None, :]].reshape(n1, -1)
        M1 = pk(T.evaluate("SD_M1", "iaklcd"))
        O2 = pk(T.evaluate("SD_O2", "iaklcd"))
        Z1 = pk(T.evaluate("SD_Z1", "iaklcd"))
        dK = (ev[av][None, :] + ev[bv][None, :] - eo[io][:, None] - eo[jo][:, None]).reshape(-1)
        self.MSD = [np.zeros_like(M1), M1, (dK[None, :] - dS[:, None]) * O2 + Z1]
        DD = T.evaluate("DD_M1", "ijabklcd")
        DD = DD[io[:, None], jo[:, None], av[None, :], bv[None, :]]
        DD = DD[:, :, io[:, None], jo[:, None], av[None, :], bv[None, :]]
        n2 = io.size * av.size
        self.MDD = [np.diag(dK).astype(np.complex128), DD.reshape(n2, n2)]
        self.n1 = n1


def explicit_matrix(order, x, B, eps_occ, eps_vir, dd_order=1, blocks=None):
    bl = blocks if blocks is not None else Blocks(B, eps_occ, eps_vir)
    if order == 2:
        x = 0.0
    M11 = bl.MSS[0] + bl.MSS[1] + bl.MSS[2] + x * bl.MSS[3]
    M12 = bl.MSD[1] + x * bl.MSD[2]
    M22 = bl.MDD[0] + (x * bl.MDD[1] if dd_order == 1 else 0.0)
    return np.block([[M11, M12], [M12.conj().T, M22]])


def sigma_ref(order, x, B, eps_occ, eps_vir, X, dd_order=1, T=None):
    """S = M X term by term (no explicit matrix), for moderate sizes."""
    T = T if T is not None else Tensors(B, eps_occ, eps_vir)
    o, v = T.o, T.v
    eo, ev = T.amp.eo, T.amp.ev
    if order == 2:
        x = 0.0
    X = np.atleast_2d(np.asarray(X, np.complex128))
    n1, n2 = dims(o, v)
    X1 = X[:, :n1].reshape(-1, o, v)
    X2f = unpack2(X[:, n1:], o, v)
    t = T.amp
    N2 = 0.25 * np.sum(np.abs(t.t1) ** 2)
    N3 = 0.5 * np.real(np.sum(t.t1.conj() * t.t2d))
    # singles-singles through the static block
    K1 = T.evaluate("SS_K1", "iajb")
    S2 = T.evaluate("SS_S2", "iajb") - N2 * np.einsum("ij,ab->iajb", np.eye(o), np.eye(v))
    Y2 = T.evaluate("SS_Y2", "iajb")
    dS = ev[None, :] - eo[:, None]
    W = 0.5 * (dS[None, None, :, :] - dS[:, :, None, None])
    M = np.einsum("ij,ab->iajb", np.eye(o), np.eye(v)) * dS[:, :, None, None] + K1 + W * S2 + Y2
    if x != 0.0:
        S3 = T.evaluate("SS_S3", "iajb") - N3 * np.einsum("ij,ab->iajb", np.eye(o), np.eye(v))
        Y3 = T.evaluate("SS_Y3a", "iajb") + T.evaluate("SS_Y3b", "iajb") - N2 * K1
        S2m, K1m = S2.reshape(n1, n1), K1.reshape(n1, n1)
        M = M + x * (W * S3 + Y3 - 0.5 * (S2m @ K1m + K1m @ S2m).reshape(o, v, o, v))
    S1 = np.einsum("iajb,njb->nia", M, X1)
    # singles <- doubles: 1/4 sum_klcd M_SD(ia; klcd) X_klcd
    for n in range(X.shape[0]):
        ext = [("klcd", X2f[n])]
        acc = 0.25 * T.evaluate("SD_M1", "ia", extra=ext)
        if x != 0.0:
            dK = (ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None])
            acc = acc + x * 0.25 * (T.evaluate("SD_O2", "ia", extra=[("klcd", X2f[n] * dK)])
                                    - dS * T.evaluate("SD_O2", "ia", extra=ext)
                                    + T.evaluate("SD_Z1", "ia", extra=ext))
        S1[n] = S1[n] + acc
    # doubles <- singles: sum_ia conj(M_SD(ia; klcd)) X_ia
    S2f = np.zeros_like(X2f)
    for n in range(X.shape[0]):
        ext = [("ia", X1[n])]
        acc = T.evaluate("SD_M1", "klcd", extra=ext, conj=True)
        if x != 0.0:
            dK = (ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None])
            acc = acc + x * (dK * T.evaluate("SD_O2", "klcd", extra=ext, conj=True)
                             - T.evaluate("SD_O2", "klcd", extra=[("ia", X1[n] * dS)], conj=True)
                             + T.evaluate("SD_Z1", "klcd", extra=ext, conj=True))
        S2f[n] = acc
    dK = (ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None])
    S2f = S2f + dK[None] * X2f
    if x != 0.0 and dd_order == 1:
        for n in range(X.shape[0]):
            S2f[n] = S2f[n] + x * 0.25 * T.evaluate("DD_M1", "ijab", extra=[("klcd", X2f[n])])
    return np.concatenate([S1.reshape(X.shape[0], -1), pack2(S2f, o, v)], axis=1)


def diagonal_ref(order, x, B, eps_occ, eps_vir, dd_order=1, T=None):
    """Exact diagonal: singles from the static block, doubles
    eps_a + eps_b - eps_i - eps_j + x (<ab||ab> + <ij||ij> - <ai||ai> - <aj||aj> - <bi||bi> - <bj||bj>)."""
    T = T if T is not None else Tensors(B, eps_occ, eps_vir)
    o, v = T.o, T.v
    n1 = o * v
    bl_ss = None
    if order == 2:
        x = 0.0
    # singles diagonal from the dense static block
    Xs = np.eye(n1 + dims(o, v)[1], dtype=np.complex128)[:n1]
    S = sigma_ref(order, x, B, eps_occ, eps_vir, Xs, dd_order=dd_order, T=T)
    d1 = np.real(np.diag(S[:, :n1]))
    del bl_ss
    eo, ev = T.amp.eo, T.amp.ev
    Jd = np.einsum("Qpp,Qqq->pq", B, B)
    Kd = np.einsum("Qpq,Qqp->pq", B, B)
    g = np.real(Jd - Kd)
    io, jo = _pairs(o)
    av, bv = _pairs(v)
    goo, gvv, gvo = g[:o, :o], g[o:, o:], g[o:, :o]
    z = ev[av][None, :] + ev[bv][None, :] - eo[io][:, None] - eo[jo][:, None]
    f = (gvv[av, bv][None, :] + goo[io, jo][:, None] - gvo[av][:, io].T - gvo[av][:, jo].T
         - gvo[bv][:, io].T - gvo[bv][:, jo].T)
    xd = x if dd_order == 1 else 0.0
    return np.concatenate([d1, (z + xd * f).ravel()])
