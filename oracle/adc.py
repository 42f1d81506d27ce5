"""Closed-form IP- and EA-ADC secular matrices and sigma products (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The ISR secular matrix ``M_IJ = <Psi~_I|H - E0|Psi~_J>`` (Sec. 2.1, Eq. 7) is
expanded in perturbation orders (Eq. 11). The paper prints no working
equations; the expressions below were derived from the ISR construction it
states (correlated excited states, Gram-Schmidt against lower classes,
symmetric orthonormalisation) with a Moller-Plesset ground state, and each
block and order is pinned element by element against the brute-force ISR
series of ``isr_series``.

Derivation outline for the lowest class (IP 1h, EA 1p): it is orthonormalised
only within itself, so ``M11 = S^-1/2 K S^-1/2`` with ``S`` the overlap of the
correlated states and ``K_pq = <Psi0| C_p^+ [H, C_q] |Psi0>``. Through third
order this gives ``M11 = M0 + Y + 1/2 (eps_p - eps_q) P`` (IP with the sign of
the hole energies) where ``P`` is the correlation part of the overlap and
``Y`` collects expectation values of the commutator's two-body part.

Basis-state phase convention (the paper's operator order, Eqs. 3-4):
  IP  1h  ``a_i |Psi0>``;  2h1p ``a+_a a_i a_j |Psi0>`` with ``i < j``;
  EA  1p  ``a+_a |Psi0>``; 2p1h ``a+_a a+_b a_j |Psi0>`` with ``a < b``.
Packed vector layout:
  IP  ``[X_i (nocc) | X_(i<j),a (npairs_o * nvir)]``, ``a`` fastest;
  EA  ``[X_a (nvir) | X_j,(a<b) (nocc * npairs_v)]``, pair fastest.
Pairs are enumerated row-major over the strict upper triangle.

Scaled third order (Sec. 2.1, Eq. 12 and the sentence after it): the paper
writes ``M0 + M1 + M2 + x M3`` and requires x = 0 to be ADC(2) and x = 1 to be
ADC(3). Every term that ADC(3) adds to ADC(2) is scaled by x: the third-order
main block, the second-order coupling and the first-order satellite block.
This keeps M linear in x, so ``d omega / d x = y^H (M_ADC3 - M_ADC2) y``.

Eigenvalues of M are E(N-1) - E0 (IP), E(N+1) - E0 (EA).
"""
from __future__ import annotations

import numpy as np

from .integrals import Amplitudes, eri

ein = np.einsum

__all__ = ["dims", "unpack2", "pack2", "Blocks", "explicit_matrix", "sigma_ref",
           "diagonal_ref", "main_block"]


def dims(kind, nocc, nvir):
    """(n1, n2) sizes of the two classes."""
    if kind == "IP":
        return nocc, nocc * (nocc - 1) // 2 * nvir
    if kind == "EA":
        return nvir, nocc * (nvir * (nvir - 1) // 2)
    raise ValueError(kind)


def unpack2(kind, X2, nocc, nvir):
    """Packed satellite amplitudes -> full antisymmetric array.

    IP: ``[k][npairs_o*nvir]`` -> ``[k, i, j, a]`` antisymmetric in (i, j).
    EA: ``[k][nocc*npairs_v]`` -> ``[k, j, a, b]`` antisymmetric in (a, b).
    """
    X2 = np.atleast_2d(X2)
    k = X2.shape[0]
    if kind == "IP":
        iu, ju = np.triu_indices(nocc, 1)
        Y = X2.reshape(k, iu.size, nvir)
        F = np.zeros((k, nocc, nocc, nvir), dtype=np.complex128)
        F[:, iu, ju, :] = Y
        F[:, ju, iu, :] = -Y
        return F
    iu, ju = np.triu_indices(nvir, 1)
    Y = X2.reshape(k, nocc, iu.size)
    F = np.zeros((k, nocc, nvir, nvir), dtype=np.complex128)
    F[:, :, iu, ju] = Y
    F[:, :, ju, iu] = -Y
    return F


def pack2(kind, F, nocc, nvir):
    """Inverse of ``unpack2`` (takes the upper-triangle elements)."""
    k = F.shape[0]
    if kind == "IP":
        iu, ju = np.triu_indices(nocc, 1)
        return F[:, iu, ju, :].reshape(k, -1)
    iu, ju = np.triu_indices(nvir, 1)
    return F[:, :, iu, ju].reshape(k, -1)


# ---------------------------------------------------------------------------
# main (lowest-class) block, orders 0, 2, 3
# ---------------------------------------------------------------------------

def main_block(kind, amp):
    """[M0, M1, M2, M3] of the 1h (IP) or 1p (EA) block.

    EA (indices a, b virtual):
      M0_ab = eps_a delta_ab,  M1 = 0,
      M2_ab = -1/2 sum_klc t_kl^ac <kl||bc> + 1/2 (eps_a - eps_b) gamma_ba,
      M3_ab = Y3_ab + 1/2 (eps_a - eps_b) gamma3_ba with
        Y3_ab = -1/2 sum_klc t2_kl^ac <kl||bc> - sum_md <ma||bd> t2_m^d
                + sum_dk <ad||bk> conj(t2_k^d) + sum_de <ad||be> gamma_de
                + 1/4 sum_ijcde <cd||be> conj(t_ij^cd) t_ij^ea
                + sum_mn <ma||bn> h_nm - sum_mcn <mc||bn> R_ca,nm,
        gamma_de = <Psi1|a+_d a_e|Psi1>, gamma3 its third-order analogue.
    IP (indices i, j occupied):
      M0_ij = -eps_i delta_ij,  M1 = 0,
      M2_ij = 1/2 sum_kcd <kj||cd> t_ik^cd - 1/2 (eps_i - eps_j) h_ji,
      M3_ij = Y3_ij - 1/2 (eps_i - eps_j) h3_ji with
        Y3_ij = 1/2 sum_kcd <kj||cd> t2_ik^cd - sum_ke <kj||ei> t2_k^e
                + sum_ck <cj||ik> conj(t2_k^c) + sum_kl <kj||li> h_lk
                + 1/4 sum <kj||lm> conj(t_lm^ef) t_ik^ef - sum_cd <cj||di> gamma_cd
                + sum <cj||dk> conj(t_kl^cf) t_il^df.
    """
    B, o = amp.B, amp.nocc
    eo, ev = amp.eo, amp.ev
    t1, t2s, t2d = amp.t1, amp.t2s, amp.t2d
    tc = t1.conj()
    if kind == "EA":
        M0 = np.diag(ev).astype(np.complex128)
        oovv = eri(B, o, "oovv")
        vvvv = eri(B, o, "vvvv")
        ovvo = eri(B, o, "ovvo")
        de = ev[:, None] - ev[None, :]
        M2 = -0.5 * ein("klac,klbc->ab", t1, oovv) + 0.5 * de * amp.gvv.T
        g3 = 0.5 * (ein("ijdf,ijef->de", tc, t2d) + ein("ijdf,ijef->de", t2d.conj(), t1))
        Y3 = (-0.5 * ein("klac,klbc->ab", t2d, oovv)
              - ein("mabd,md->ab", eri(B, o, "ovvv"), t2s)
              + ein("adbk,kd->ab", eri(B, o, "vvvo"), t2s.conj())
              + ein("adbe,de->ab", vvvv, amp.gvv)
              + 0.25 * ein("cdbe,ijcd,ijea->ab", vvvv, tc, t1, optimize=True)
              + ein("mabn,nm->ab", ovvo, amp.hoo)
              - ein("mcbn,canm->ab", ovvo, amp.R))
        M3 = Y3 + 0.5 * de * g3.T
        return [M0, np.zeros_like(M0), M2, M3]
    if kind == "IP":
        M0 = np.diag(-eo).astype(np.complex128)
        oovv = eri(B, o, "oovv")
        oooo = eri(B, o, "oooo")
        vovo = eri(B, o, "vovo")
        do = eo[:, None] - eo[None, :]
        M2 = 0.5 * ein("kjcd,ikcd->ij", oovv, t1) - 0.5 * do * amp.hoo.T
        h3 = 0.5 * (ein("jkcd,ikcd->ji", tc, t2d) + ein("jkcd,ikcd->ji", t2d.conj(), t1))
        Y3 = (0.5 * ein("kjcd,ikcd->ij", oovv, t2d)
              - ein("kjei,ke->ij", eri(B, o, "oovo"), t2s)
              + ein("cjik,kc->ij", eri(B, o, "vooo"), t2s.conj())
              + ein("kjli,lk->ij", oooo, amp.hoo)
              + 0.25 * ein("kjlm,lmef,ikef->ij", oooo, tc, t1, optimize=True)
              - ein("cjdi,cd->ij", vovo, amp.gvv)
              + ein("cjdk,klcf,ildf->ij", vovo, tc, t1, optimize=True))
        M3 = Y3 - 0.5 * do * h3.T
        return [M0, np.zeros_like(M0), M2, M3]
    raise ValueError(kind)


class Blocks:
    """All order-resolved blocks of IP/EA-ADC(3) for a small case (dense)."""

    def __init__(self, kind, B, eps_occ, eps_vir):
        self.kind = kind
        amp = Amplitudes(B, eps_occ, eps_vir)
        self.amp = amp
        o, v = amp.nocc, amp.nvir
        eo, ev = amp.eo, amp.ev
        tc = amp.t1.conj()
        self.M11 = main_block(kind, amp)
        if kind == "EA":
            iu, ju = np.triu_indices(v, 1)
            c1 = eri(B, o, "vovv")  # <ck||de>  [c, k, d, e]
            c2 = (0.5 * ein("ckmn,mnde->ckde", eri(B, o, "vooo"), tc)
                  + ein("cgem,kmgd->ckde", eri(B, o, "vvvo"), tc)
                  - ein("cgdm,kmge->ckde", eri(B, o, "vvvo"), tc))
            self.M12 = [np.zeros((v, o * iu.size), np.complex128),
                        c1[:, :, iu, ju].reshape(v, -1), c2[:, :, iu, ju].reshape(v, -1)]
            vvvv = eri(B, o, "vvvv")
            vovo = eri(B, o, "vovo")  # <ak||cj>  [a, k, c, j]
            dk, dv = np.eye(o), np.eye(v)
            s1 = (ein("jk,abcd->jabkcd", dk, vvvv)
                  - ein("bd,akcj->jabkcd", dv, vovo) + ein("ad,bkcj->jabkcd", dv, vovo)
                  + ein("bc,akdj->jabkcd", dv, vovo) - ein("ac,bkdj->jabkcd", dv, vovo))
            n2 = o * iu.size
            s1 = s1[:, iu, ju][:, :, :, iu, ju].reshape(n2, n2)
            d0 = (ev[iu][None, :] + ev[ju][None, :] - eo[:, None]).ravel()
        elif kind == "IP":
            iu, ju = np.triu_indices(o, 1)
            c1 = eri(B, o, "oovo").transpose(3, 1, 0, 2)  # <ji||ak> -> [k, i, j, a]
            c2 = (0.5 * ein("efak,jief->kija", eri(B, o, "vvvo"), tc)
                  - ein("fimk,jmfa->kija", eri(B, o, "vooo"), tc)
                  + ein("fjmk,imfa->kija", eri(B, o, "vooo"), tc))
            self.M12 = [np.zeros((o, iu.size * v), np.complex128),
                        c1[:, iu, ju, :].reshape(o, -1), c2[:, iu, ju, :].reshape(o, -1)]
            oooo = eri(B, o, "oooo")
            vovo = eri(B, o, "vovo")  # <ak||bi>  [a, k, b, i]
            do, dv = np.eye(o), np.eye(v)
            s1 = (ein("ab,klij->ijaklb", dv, oooo)
                  - ein("jl,akbi->ijaklb", do, vovo) + ein("il,akbj->ijaklb", do, vovo)
                  + ein("jk,albi->ijaklb", do, vovo) - ein("ik,albj->ijaklb", do, vovo))
            n2 = iu.size * v
            s1 = s1[iu, ju][:, :, iu, ju].reshape(n2, n2)
            d0 = (ev[None, :] - eo[iu][:, None] - eo[ju][:, None]).ravel()
        else:
            raise ValueError(kind)
        self.M22 = [np.diag(d0).astype(np.complex128), s1]
        self.n1 = self.M11[0].shape[0]


def explicit_matrix(kind, order, x, B, eps_occ, eps_vir, blocks=None):
    """Dense Hermitian M for ADC(2) (order=2) or ADC(2)+x(3) (order=3)."""
    bl = blocks if blocks is not None else Blocks(kind, B, eps_occ, eps_vir)
    if order == 2:
        x = 0.0
    elif order != 3:
        raise ValueError("order must be 2 or 3")
    M11 = bl.M11[0] + bl.M11[2] + x * bl.M11[3]
    M12 = bl.M12[1] + x * bl.M12[2]
    M22 = bl.M22[0] + x * bl.M22[1]
    top = np.concatenate([M11, M12], axis=1)
    bot = np.concatenate([M12.conj().T, M22], axis=1)
    return np.concatenate([top, bot], axis=0)


# ---------------------------------------------------------------------------
# matrix-free sigma
# ---------------------------------------------------------------------------

def sigma_ref(kind, order, x, B, eps_occ, eps_vir, X, amp=None, M11=None):
    """S = M X for a [k][N] block of vectors, term by term (no explicit M).

    EA (X1_a, X2_j,ab full antisymmetric):
      S1_c  = sum_b M11_cb X1_b + 1/2 sum_kde (<ck||de> + x M12^(2)_c,kde) X2_kde
      S2_kde = sum_c conj(<ck||de> + x M12^(2)_c,kde) X1_c
               + (eps_d + eps_e - eps_k) X2_kde
               + x [ 1/2 sum_fg <de||fg> X2_kfg - P(de) sum_lf <dl||fk> X2_lfe ]
    IP (X1_k, X2_ija full antisymmetric in ij):
      S1_k  = sum_l M11_kl X1_l + 1/2 sum_ija (<ji||ak> + x M12^(2)_k,ija) X2_ija
      S2_ija = sum_k conj(...) X1_k + (eps_a - eps_i - eps_j) X2_ija
               + x [ 1/2 sum_kl <kl||ij> X2_kla + P(ij) sum_kb <ak||bj> X2_kib ]
    ADC(2) (order=2) drops every x term and the third-order main block.
    """
    X = np.atleast_2d(np.asarray(X, dtype=np.complex128))
    amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir, second_order=(order == 3))
    o, v = amp.nocc, amp.nvir
    eo, ev = amp.eo, amp.ev
    if order == 2:
        x = 0.0
    n1, n2 = dims(kind, o, v)
    X1 = X[:, :n1]
    X2f = unpack2(kind, X[:, n1:], o, v)
    tc = amp.t1.conj()
    if M11 is None:
        mb = main_block(kind, amp) if order == 3 else None
        if order == 3:
            M11 = mb[0] + mb[2] + x * mb[3]
        else:
            M11 = _main_block_order2(kind, amp)
    S1 = X1 @ M11.T
    if kind == "EA":
        vovv = eri(B, o, "vovv")  # <ck||de>
        c2 = (0.5 * ein("ckmn,mnde->ckde", eri(B, o, "vooo"), tc)
              + ein("cgem,kmgd->ckde", eri(B, o, "vvvo"), tc)
              - ein("cgdm,kmge->ckde", eri(B, o, "vvvo"), tc)) if x != 0.0 else 0.0
        C = vovv + x * c2
        S1 = S1 + 0.5 * ein("ckde,nkde->nc", C, X2f)
        S2 = ein("ckde,nc->nkde", np.conj(C), X1)
        dd = ev[None, :, None] + ev[None, None, :] - eo[:, None, None]
        S2 = S2 + dd[None] * X2f
        if x != 0.0:
            S2 = S2 + x * 0.5 * ein("defg,nkfg->nkde", eri(B, o, "vvvv"), X2f)
            ring = ein("dlfk,nlfe->nkde", eri(B, o, "vovo"), X2f)
            S2 = S2 - x * (ring - ring.transpose(0, 1, 3, 2))
    elif kind == "IP":
        c1 = eri(B, o, "oovo").transpose(3, 1, 0, 2)  # [k, i, j, a]
        c2 = (0.5 * ein("efak,jief->kija", eri(B, o, "vvvo"), tc)
              - ein("fimk,jmfa->kija", eri(B, o, "vooo"), tc)
              + ein("fjmk,imfa->kija", eri(B, o, "vooo"), tc)) if x != 0.0 else 0.0
        C = c1 + x * c2
        S1 = S1 + 0.5 * ein("kija,nija->nk", C, X2f)
        S2 = ein("kija,nk->nija", np.conj(C), X1)
        dd = ev[None, None, :] - eo[:, None, None] - eo[None, :, None]
        S2 = S2 + dd[None] * X2f
        if x != 0.0:
            S2 = S2 + x * 0.5 * ein("klij,nkla->nija", eri(B, o, "oooo"), X2f)
            ring = ein("akbj,nkib->nija", eri(B, o, "vovo"), X2f)
            S2 = S2 + x * (ring - ring.transpose(0, 2, 1, 3))
    else:
        raise ValueError(kind)
    return np.concatenate([S1, pack2(kind, S2, o, v)], axis=1)


def _main_block_order2(kind, amp):
    B, o = amp.B, amp.nocc
    if kind == "EA":
        de = amp.ev[:, None] - amp.ev[None, :]
        return (np.diag(amp.ev) - 0.5 * ein("klac,klbc->ab", amp.t1, eri(B, o, "oovv"))
                + 0.5 * de * amp.gvv.T)
    do = amp.eo[:, None] - amp.eo[None, :]
    return (np.diag(-amp.eo) + 0.5 * ein("kjcd,ikcd->ij", eri(B, o, "oovv"), amp.t1)
            - 0.5 * do * amp.hoo.T)


def diagonal_ref(kind, order, x, B, eps_occ, eps_vir, amp=None):
    """Exact diagonal of M (real), packed layout.

    Satellite diagonal: EA ``eps_a + eps_b - eps_j + x(<ab||ab> - <aj||aj> - <bj||bj>)``;
    IP ``eps_a - eps_i - eps_j + x(<ij||ij> - <ai||ai> - <aj||aj>)``.
    """
    amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir, second_order=(order == 3))
    o, v = amp.nocc, amp.nvir
    eo, ev = amp.eo, amp.ev
    if order == 2:
        x = 0.0
        M11 = _main_block_order2(kind, amp)
    else:
        mb = main_block(kind, amp)
        M11 = mb[0] + mb[2] + x * mb[3]
    d1 = np.real(np.diag(M11))
    nmo = o + v
    # <pq||pq> for all p, q from Eq. 43
    Jd = ein("Qpp,Qqq->pq", B, B)
    Kd = ein("Qpq,Qqp->pq", B, B)
    g = np.real(Jd - Kd)
    if kind == "EA":
        iu, ju = np.triu_indices(v, 1)
        gvv = g[o:, o:]
        gvo = g[o:, :o]
        d2 = (ev[iu][None, :] + ev[ju][None, :] - eo[:, None]
              + x * (gvv[iu, ju][None, :] - gvo[iu, :].T - gvo[ju, :].T))
    else:
        iu, ju = np.triu_indices(o, 1)
        goo = g[:o, :o]
        gvo = g[o:, :o]
        d2 = (ev[None, :] - eo[iu][:, None] - eo[ju][:, None]
              + x * (goo[iu, ju][:, None] - gvo[:, iu].T - gvo[:, ju].T))
    return np.concatenate([d1, d2.ravel()])
