"""State-specific frozen natural spinors (oracle), Sec. 2.4, Eqs. 31-32.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For root k of EA- or EE-ADC(2) with eigenvector y, the state's virtual
density is taken in the zeroth-order intermediate-state representation: the
excited configurations themselves, weighted by the ADC(2) amplitudes,

  EA  |Psi> = sum_a y_a a+_a |Phi> + sum_{j, a<b} y_jab a+_a a+_b a_j |Phi>,
  EE  |Psi> = sum_ia y_ia a+_a a_i |Phi> + sum_{i<j, a<b} y_ijab a+_a a+_b a_j a_i |Phi>,

and D^state_ab = <Psi| a+_b a_a |Psi> for virtual a, b, the index order of
Eq. 25 (there D^MP2_ab = 1/2 sum_ijc t_ij^ac conj(t_ij^bc) = <Psi1| a+_b a_a |Psi1>).
Wick's theorem gives, with the doubles Y as full antisymmetric arrays,

  EA  D_ab = y_a conj(y_b) + sum_{j,c} Y_jac conj(Y_jbc),
  EE  D_ab = sum_i y_ia conj(y_ib) + 1/2 sum_{ijc} Y_ijac conj(Y_ijbc)

(pinned against the same expectation value in determinant space). Eq. 31:
D^SS = D^MP2 + D^state; Eqs. 26-30 on D^SS give U = V~ Z~ and eps~.

The canonical eigenvector is carried into the truncated basis through the
virtual creation operators: with a+'_a' = sum_a U_aa' a+_a, a+_a = sum_a'
conj(U_aa') a+'_a' on the kept span, so y'_a' = sum_a conj(U_aa') y_a on every
virtual index. It is the guess of the root-specific solves, which take the
eigenpair of the truncated-basis matrix with the largest |<y'|x>|. Eq. 32:
omega_corrected = omega3_fns + omega2_canonical - omega2_fns.
"""
from __future__ import annotations

import numpy as np

from . import adc as _adc
from . import adc_ee as _ee
from .fns import fns_basis, fns_density, transform_cholesky

__all__ = ["state_density", "to_fns_basis", "follow_root", "ssfns", "matrix"]


def matrix(kind, order, x, B, eps_occ, eps_vir):
    """Explicit ADC matrix (small cases)."""
    if kind == "EE":
        return _ee.explicit_matrix(order, x, B, eps_occ, eps_vir)
    return _adc.explicit_matrix(kind, order, x, B, eps_occ, eps_vir)


def _split(kind, y, nocc, nvir):
    """Singles (full) and doubles (full antisymmetric) parts of a packed vector."""
    y = np.asarray(y, np.complex128).reshape(-1)
    if kind == "EA":
        n1 = nvir
        return y[:n1], _adc.unpack2("EA", y[n1:][None, :], nocc, nvir)[0]
    if kind == "EE":
        n1 = nocc * nvir
        return y[:n1].reshape(nocc, nvir), _ee.unpack2(y[n1:][None, :], nocc, nvir)[0]
    raise ValueError("state density: EA or EE")


def state_density(kind, y, nocc, nvir):
    """D^state_ab = <Psi| a+_b a_a |Psi> of the configurations weighted by y."""
    y1, Y = _split(kind, y, nocc, nvir)
    if kind == "EA":
        return np.outer(y1, y1.conj()) + np.einsum("jac,jbc->ab", Y, Y.conj())
    return np.einsum("ia,ib->ab", y1, y1.conj()) + 0.5 * np.einsum("ijac,ijbc->ab", Y, Y.conj())


def to_fns_basis(kind, y, nocc, nvir, U):
    """y' with y'_a' = sum_a conj(U_aa') y_a on every virtual index, packed."""
    y1, Y = _split(kind, y, nocc, nvir)
    Uc = U.conj()
    nk = U.shape[1]
    if kind == "EA":
        g1 = Uc.T @ y1
        G = np.einsum("aA,bB,jab->jAB", Uc, Uc, Y)
        return np.concatenate([g1, _adc.pack2("EA", G[None], nocc, nk)[0]])
    g1 = y1 @ Uc
    G = np.einsum("aA,bB,ijab->ijAB", Uc, Uc, Y)
    return np.concatenate([g1.reshape(-1), _ee.pack2(G[None], nocc, nk)[0]])


def follow_root(M, guess):
    """Eigenpair of the Hermitian M with the largest overlap |<guess|x>|."""
    w, V = np.linalg.eigh(M)
    ov = np.abs(V.conj().T @ guess)
    r = int(np.argmax(ov))
    return float(w[r]), V[:, r], r, float(ov[r] / max(np.linalg.norm(guess), 1e-300))


def ssfns(kind, order, x, B, eps_occ, eps_vir, nroots, eta_crit):
    """Per root: corrected SS-FNS energy (Eq. 32) and its parts, from explicit matrices."""
    eo = np.asarray(eps_occ, np.float64)
    ev = np.asarray(eps_vir, np.float64)
    o, v = eo.shape[0], ev.shape[0]
    M2 = matrix(kind, 2, 0.0, B, eo, ev)
    w2, V2 = np.linalg.eigh(M2)
    Dmp2 = fns_density(B, eo, ev)
    out = []
    for k in range(nroots):
        y = V2[:, k]
        D = Dmp2 + state_density(kind, y, o, v)
        eta, _, nk, U, et = fns_basis(D, ev, eta_crit)
        Bn = transform_cholesky(B, o, U)
        g = to_fns_basis(kind, y, o, v, U)
        g = g / np.linalg.norm(g)
        wa, _, ra, oa = follow_root(matrix(kind, 2, 0.0, Bn, eo, et), g)
        wb, _, rb, ob = follow_root(matrix(kind, order, x, Bn, eo, et), g)
        out.append({"omega_corrected": wb + float(w2[k]) - wa, "omega_fns": wb, "omega2_canonical": float(w2[k]),
                    "omega2_fns": wa, "n_keep": int(nk), "root2": ra, "root3": rb, "overlap2": oa,
                    "overlap3": ob, "eta": eta, "eps_new": et, "U": U})
    return out
