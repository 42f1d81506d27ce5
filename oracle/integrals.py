"""Antisymmetrised integrals, Moller-Plesset amplitudes and densities (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions
-----------
* Spinors are numbered occupied first: ``0..nocc-1`` occupied (i, j, k, ...),
  ``nocc..nmo-1`` virtual (a, b, c, ...).
* ``B[Q, p, q]`` are the Cholesky vectors in the spinor basis, Hermitian in
  ``(p, q)`` (Eq. 42 of a Hermitian ERI matrix).
* ``<pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr)`` (Eq. 43), no complex conjugate
  anywhere; the Hermiticity of each ``B[Q]`` makes ``<rs||pq> = conj <pq||rs>``.
* The Hamiltonian is ``sum h_pq a+p a_q + 1/4 sum <pq||rs> a+p a+q a_s a_r``
  with a canonical Hartree-Fock reference, Fock matrix ``diag(eps)``.
* First-order doubles ``t_ij^ab = <ab||ij> / D_ij^ab``,
  ``D_ij^ab = eps_i + eps_j - eps_a - eps_b`` (the denominators of Eq. 25);
  ``Psi1 = 1/4 sum t_ij^ab a+a a+b a_j a_i |Phi>``.
* Arrays are stored with occupied indices first: ``t[i, j, a, b]``.
"""
from __future__ import annotations

import numpy as np

ein = np.einsum

__all__ = ["eri", "Amplitudes", "semicanonical"]


def eri(B, nocc, spec):
    """Block of <pq||rs> (Eq. 43) selected by a 4-letter spec over {'o','v'}.

    ``spec = 'vvoo'`` returns ``g[a, b, i, j] = <ab||ij>``.
    """
    nmo = B.shape[1]
    sl = {"o": slice(0, nocc), "v": slice(nocc, nmo)}
    p, q, r, s = (sl[c] for c in spec)
    return (ein("Qpr,Qqs->pqrs", B[:, p, r], B[:, q, s])
            - ein("Qps,Qqr->pqrs", B[:, p, s], B[:, q, r]))


class Amplitudes:
    """Perturbative ground-state quantities needed by ADC up to third order.

    t1   first-order doubles t_ij^ab                        [i, j, a, b]
    t2s  second-order singles t_i^a                         [i, a]
    t2d  second-order doubles t_ij^ab                       [i, j, a, b]
    gvv  second-order <Psi1|a+_d a_e|Psi1>                  [d, e]
    hoo  second-order <Psi1|a_n a+_m|Psi1> (hole density)   [n, m]
    R    <Psi1|a+_c a_n a+_m a_a|Psi1>                      [c, a, n, m]

    Second-order amplitudes follow Rayleigh-Schroedinger theory with the
    normal-ordered fluctuation potential:
      (eps_i - eps_a) t_i^a = 1/2 sum_jcd <aj||cd> t_ij^cd
                              - 1/2 sum_jkc <jk||ic> t_jk^ac,
      D_ij^ab t2_ij^ab = 1/2 sum_cd <ab||cd> t_ij^cd + 1/2 sum_kl <kl||ij> t_kl^ab
                         + P(ij)P(ab) sum_kc <kb||cj> t_ik^ac.
    """

    def __init__(self, B, eps_occ, eps_vir, second_order=True):
        eo = np.asarray(eps_occ, dtype=np.float64)
        ev = np.asarray(eps_vir, dtype=np.float64)
        o = eo.shape[0]
        self.nocc, self.nvir = o, ev.shape[0]
        self.B, self.eo, self.ev = B, eo, ev
        D2 = (eo[:, None, None, None] + eo[None, :, None, None]
              - ev[None, None, :, None] - ev[None, None, None, :])
        self.D2 = D2
        self.t1 = eri(B, o, "vvoo").transpose(2, 3, 0, 1) / D2
        t1 = self.t1
        tc = t1.conj()
        self.gvv = 0.5 * ein("ijdf,ijef->de", tc, t1)
        self.hoo = 0.5 * ein("njef,mjef->nm", tc, t1)
        if not second_order:
            return
        D1 = eo[:, None] - ev[None, :]
        self.t2s = (0.5 * ein("ajcd,ijcd->ia", eri(B, o, "vovv"), t1)
                    - 0.5 * ein("jkic,jkac->ia", eri(B, o, "ooov"), t1)) / D1
        ring = ein("kbcj,ikac->ijab", eri(B, o, "ovvo"), t1)
        ring = (ring - ring.transpose(1, 0, 2, 3) - ring.transpose(0, 1, 3, 2)
                + ring.transpose(1, 0, 3, 2))
        self.t2d = (0.5 * ein("abcd,ijcd->ijab", eri(B, o, "vvvv"), t1)
                    + 0.5 * ein("klij,klab->ijab", eri(B, o, "oooo"), t1)
                    + ring) / D2
        self.R = ein("njcf,mjaf->canm", tc, t1)

    def mp2_energy(self):
        """E2 = 1/4 sum_ijab <ij||ab> t_ij^ab."""
        return 0.25 * ein("ijab,ijab->", eri(self.B, self.nocc, "oovv"), self.t1)


def semicanonical(F_occ, F_vir, B):
    """Problem in the semicanonical basis, from full Fock blocks.

    The method takes a diagonal Fock matrix. A reference whose occupied-occupied
    and virtual-virtual Fock blocks are not diagonal (a rotated basis) is
    brought to that form as the natural-spinor basis is in Sec. 2.4 (Eq. 29):
    each block is diagonalised on its own, F_oo Z_o = Z_o eps_o and
    F_vv Z_v = Z_v eps_v (eigenvalues ascending), and the Cholesky vectors
    follow the same rotation W = diag(Z_o, Z_v) as in Eq. 42:
    B'[Q] = W^H B[Q] W. Returns (eps_occ, eps_vir, B').
    """
    eo, Zo = np.linalg.eigh(np.asarray(F_occ))
    ev, Zv = np.linalg.eigh(np.asarray(F_vir))
    o, v = Zo.shape[0], Zv.shape[0]
    W = np.zeros((o + v, o + v), dtype=np.complex128)
    W[:o, :o] = Zo
    W[o:, o:] = Zv
    Bs = ein("pi,Qpq,qj->Qij", W.conj(), B, W)
    return eo, ev, Bs
