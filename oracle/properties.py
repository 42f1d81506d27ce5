"""Ground-to-excited transition densities of EE-ADC (oracle), Sec. 2.2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The transition density of state K is rho_pq = <Psi_K| a+_p a_q |Psi0> =
sum_I conj(Y_IK) f_I(pq), with the ISR transition moments
f_I(pq) = <Psi~_I| a+_p a_q |Psi0> (Psi~_I the intermediate states of Eqs.
5-6, Psi0 the normalised MP ground state); a transition moment of a
one-particle operator d is T = sum_pq d_pq rho_pq.

Through the orders used with ADC(2) and ADC(3) eigenvectors (singles to
second, doubles to first order), with S the singles label (i, a), D the
doubles label (i<j, a<b), t / t2 the first- / second-order doubles
amplitudes, s2 the second-order singles and S2 the second-order overlap of
the orthogonalised singles precursors (the singles f is S^{1/2} on its
excitation block):

  f_S(b, j) = d_ab d_ij + 1/2 S2_{ia,jb}           (p = b virtual, q = j occupied)
  f_S(j, b) = t_ij^ab + t2_ij^ab                    (p = j occupied, q = b virtual)
  f_S(k, l) = -d_li s2_k^a,    f_S(e, f) = d_ae s2_i^f
  f_D(k, l) = -d_li t_kj^ab - d_lj t_ik^ab,    f_D(e, f) = d_ae t_ij^fb + d_be t_ij^af

(every term pinned against the brute-force ISR series in determinant space).
Summed over the packed doubles with the full antisymmetric Y:

  rho_bj = conj(y_jb) + 1/2 sum_ia conj(y_ia) S2_{ia,jb}
  rho_jb = sum_ia conj(y_ia) (t_ij^ab + t2_ij^ab)
  rho_kl = -sum_a conj(y_la) s2_k^a - 1/2 sum_jab conj(Y_ljab) t_kj^ab
  rho_ef = sum_i conj(y_ie) s2_i^f + 1/2 sum_ijb conj(Y_ijeb) t_ij^fb

Excited-state density (the level the paper states for ADC(2) states: the
ground-state density through second order plus the zeroth-order
intermediate-state representation of D - D0, i.e. the configurations
weighted by the eigenvector), rho^K_pq = <a+_p a_q>:

  ground state  rho0_ij = d_ij - 1/2 sum_kab conj(t_jk^ab) t_ik^ab,
                rho0_ab = 1/2 sum_ijc conj(t_ij^ac) t_ij^bc,
                rho0_jb = s2_j^b,  rho0_bj = conj(s2_j^b);
  difference    rho_kl += -sum_a conj(y_la) y_ka - 1/2 sum_jab conj(Y_ljab) Y_kjab,
                rho_ef += sum_i conj(y_ie) y_if + 1/2 sum_ijc conj(Y_ijec) Y_ijfc,
                rho_jb += sum_ia conj(y_ia) Y_ijab,  rho_bj += sum_ia conj(Y_ijab) y_ia
(pinned against the same quantities in determinant space).

Spectroscopic amplitudes of IP/EA states (the ISR transition moments of the
one-particle operators a_p / a+_p), x_p = <Psi_n| a_p |Psi0> (IP) or
<Psi_n| a+_p |Psi0> (EA) = sum_I conj(Y_In) f_I(p), main class through second
and satellite class through first order (the same orders as the EE moments):

  IP, main i:        f_i(k) = d_ik - 1/4 sum_jab conj(t_kj^ab) t_ij^ab,  f_i(b) = s2_i^b
  IP, sat (i<j, a):  f(b) = t_ij^ab
  EA, main a:        f_a(b) = d_ab - 1/4 sum_ijc conj(t_ij^bc) t_ij^ac,  f_a(k) = -s2_k^a
  EA, sat (j, a<b):  f(k) = t_jk^ab

so, with Y the satellite amplitudes as a full antisymmetric array,

  IP  x_k = conj(y_k) - 1/4 sum_ijab conj(y_i) conj(t_kj^ab) t_ij^ab
      x_b = sum_i conj(y_i) s2_i^b + 1/2 sum_ija conj(Y_ija) t_ij^ab
  EA  x_b = conj(y_b) - 1/4 sum_aijc conj(y_a) conj(t_ij^bc) t_ij^ac
      x_k = -sum_a conj(y_a) s2_k^a + 1/2 sum_jab conj(Y_jab) t_jk^ab
(pinned against the brute-force (N-1)/(N+1)-electron ISR series).

State and state-to-state one-particle densities of all three kinds at the
level of the excited-state density above, rho^KL_pq = <Psi_K| a+_p a_q |Psi_L>
= (y_K^H y_L) rho0_pq + (the configurations' difference density between K and
L), with the configuration blocks (K on the bra, L on the ket, Y the class-2
amplitudes as a full antisymmetric array):

  EE  kl: -sum_a conj(yK_la) yL_ka - 1/2 sum_jab conj(YK_ljab) YL_kjab
      ef:  sum_i conj(yK_ie) yL_if + 1/2 sum_ijc conj(YK_ijec) YL_ijfc
      jb:  sum_ia conj(yK_ia) YL_ijab,   bj: sum_ia conj(YK_ijab) yL_ia
  IP  kl: -conj(yK_l) yL_k - sum_ja conj(YK_lja) YL_kja
      ab:  1/2 sum_ij conj(YK_ija) YL_ijb
      jb: -sum_i conj(yK_i) YL_ijb,      bj: -sum_i conj(YK_ijb) yL_i
  EA  kl: -1/2 sum_ab conj(YK_lab) YL_kab
      ab:  conj(yK_a) yL_b + sum_jc conj(YK_jac) YL_jbc
      jb:  sum_a conj(yK_a) YL_jab,      bj: sum_a conj(YK_jab) yL_a
(pinned against the same matrix elements in determinant space).
"""
from __future__ import annotations

import numpy as np

from . import adc as _ipea
from . import adc_ee as _ee
from .integrals import Amplitudes

__all__ = ["singles_overlap2", "transition_density", "transition_moment", "excited_state_density",
           "spectroscopic_amplitudes", "ground_state_density", "state_pair_density"]


def singles_overlap2(B, eps_occ, eps_vir, amp=None):
    """S2_{ia,jb}: second-order overlap of the orthogonalised singles precursors."""
    T = _ee.Tensors(B, eps_occ, eps_vir, amp=amp)
    o, v = T.o, T.v
    N2 = 0.25 * np.sum(np.abs(T.amp.t1) ** 2)
    return T.evaluate("SS_S2", "iajb") - N2 * np.einsum("ij,ab->iajb", np.eye(o), np.eye(v))


def transition_density(y, B, eps_occ, eps_vir, amp=None, S2=None):
    """rho [nmo][nmo] of one EE vector y (packed singles + doubles)."""
    amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir)
    o, v = amp.nocc, amp.nvir
    S2 = S2 if S2 is not None else singles_overlap2(B, eps_occ, eps_vir, amp=amp)
    y = np.asarray(y, np.complex128).reshape(-1)
    n1 = o * v
    y1c = y[:n1].reshape(o, v).conj()
    Yc = _ee.unpack2(y[n1:][None], o, v)[0].conj()
    t, t2, s2 = amp.t1, amp.t2d, amp.t2s
    rho = np.zeros((o + v, o + v), np.complex128)
    rho[o:, :o] = y1c.T + 0.5 * np.einsum("ia,iajb->bj", y1c, S2)
    rho[:o, o:] = np.einsum("ia,ijab->jb", y1c, t + t2)
    rho[:o, :o] = -np.einsum("la,ka->kl", y1c, s2) - 0.5 * np.einsum("ljab,kjab->kl", Yc, t)
    rho[o:, o:] = np.einsum("ie,if->ef", y1c, s2) + 0.5 * np.einsum("ijeb,ijfb->ef", Yc, t)
    return rho


def transition_moment(rho, d):
    """T = sum_pq d_pq rho_pq for a one-particle operator d [nmo][nmo] (or [3][nmo][nmo])."""
    return np.einsum("...pq,pq->...", np.asarray(d), rho)


def excited_state_density(y, B, eps_occ, eps_vir, amp=None):
    """rho^K [nmo][nmo] of one EE vector y: ground state to second order + zeroth-order ISR difference."""
    amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir)
    o, v = amp.nocc, amp.nvir
    y = np.asarray(y, np.complex128).reshape(-1)
    n1 = o * v
    y1 = y[:n1].reshape(o, v)
    Y = _ee.unpack2(y[n1:][None], o, v)[0]
    t, s2 = amp.t1, amp.t2s
    rho = np.zeros((o + v, o + v), np.complex128)
    rho[:o, :o] = np.eye(o) - 0.5 * np.einsum("jkab,ikab->ij", t.conj(), t)
    rho[o:, o:] = 0.5 * np.einsum("ijac,ijbc->ab", t.conj(), t)
    rho[:o, o:] = s2
    rho[o:, :o] = s2.conj().T
    rho[:o, :o] += -np.einsum("la,ka->kl", y1.conj(), y1) - 0.5 * np.einsum("ljab,kjab->kl", Y.conj(), Y)
    rho[o:, o:] += np.einsum("ie,if->ef", y1.conj(), y1) + 0.5 * np.einsum("ijec,ijfc->ef", Y.conj(), Y)
    rho[:o, o:] += np.einsum("ia,ijab->jb", y1.conj(), Y)
    rho[o:, :o] += np.einsum("ijab,ia->bj", Y.conj(), y1)
    return rho


def spectroscopic_amplitudes(y, kind, B, eps_occ, eps_vir, amp=None):
    """x [nmo] of one IP or EA vector y (packed main + satellite)."""
    amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir)
    o, v = amp.nocc, amp.nvir
    n1, _ = _ipea.dims(kind, o, v)
    y = np.asarray(y, np.complex128).reshape(-1)
    y1c = y[:n1].conj()
    Yc = _ipea.unpack2(kind, y[n1:][None], o, v)[0].conj()
    t, s2 = amp.t1, amp.t2s
    x = np.zeros(o + v, np.complex128)
    if kind == "IP":
        x[:o] = y1c - 0.25 * np.einsum("i,kjab,ijab->k", y1c, t.conj(), t)
        x[o:] = np.einsum("i,ib->b", y1c, s2) + 0.5 * np.einsum("ija,ijab->b", Yc, t)
    elif kind == "EA":
        x[o:] = y1c - 0.25 * np.einsum("a,ijbc,ijac->b", y1c, t.conj(), t)
        x[:o] = -np.einsum("a,ka->k", y1c, s2) + 0.5 * np.einsum("jab,jkab->k", Yc, t)
    else:
        raise ValueError(kind)
    return x


def ground_state_density(amp):
    """rho0 [nmo][nmo]: the MP ground-state density through second order."""
    o, v = amp.nocc, amp.nvir
    t, s2 = amp.t1, amp.t2s
    rho = np.zeros((o + v, o + v), np.complex128)
    rho[:o, :o] = np.eye(o) - 0.5 * np.einsum("jkab,ikab->ij", t.conj(), t)
    rho[o:, o:] = 0.5 * np.einsum("ijac,ijbc->ab", t.conj(), t)
    rho[:o, o:] = s2
    rho[o:, :o] = s2.conj().T
    return rho


def _classes(kind, y, o, v):
    if kind == "EE":
        n1 = o * v
        return y[:n1].reshape(o, v), _ee.unpack2(y[n1:][None], o, v)[0]
    n1, _ = _ipea.dims(kind, o, v)
    return y[:n1], _ipea.unpack2(kind, y[n1:][None], o, v)[0]


def state_pair_density(yK, yL, kind, B, eps_occ, eps_vir, amp=None):
    """rho^KL [nmo][nmo] = <Psi_K| a+_p a_q |Psi_L> of two vectors of one kind."""
    amp = amp if amp is not None else Amplitudes(B, eps_occ, eps_vir)
    o, v = amp.nocc, amp.nvir
    yK = np.asarray(yK, np.complex128).reshape(-1)
    yL = np.asarray(yL, np.complex128).reshape(-1)
    aK, YK = _classes(kind, yK, o, v)
    aL, YL = _classes(kind, yL, o, v)
    aKc, YKc = aK.conj(), YK.conj()
    e = np.einsum
    d = np.zeros((o + v, o + v), np.complex128)
    if kind == "EE":
        d[:o, :o] = -e("la,ka->kl", aKc, aL) - 0.5 * e("ljab,kjab->kl", YKc, YL)
        d[o:, o:] = e("ie,if->ef", aKc, aL) + 0.5 * e("ijec,ijfc->ef", YKc, YL)
        d[:o, o:] = e("ia,ijab->jb", aKc, YL)
        d[o:, :o] = e("ijab,ia->bj", YKc, aL)
    elif kind == "IP":
        d[:o, :o] = -e("l,k->kl", aKc, aL) - e("lja,kja->kl", YKc, YL)
        d[o:, o:] = 0.5 * e("ija,ijb->ab", YKc, YL)
        d[:o, o:] = -e("i,ijb->jb", aKc, YL)
        d[o:, :o] = -e("ijb,i->bj", YKc, aL)
    elif kind == "EA":
        d[:o, :o] = -0.5 * e("lab,kab->kl", YKc, YL)
        d[o:, o:] = e("a,b->ab", aKc, aL) + e("jac,jbc->ab", YKc, YL)
        d[:o, o:] = e("a,jab->jb", aKc, YL)
        d[o:, :o] = e("jab,a->bj", YKc, aL)
    else:
        raise ValueError(kind)
    return np.vdot(yK, yL) * ground_state_density(amp) + d
