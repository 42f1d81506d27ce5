"""Frozen natural spinors from the MP2 virtual density (oracle), Eqs. 25-30.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Steps, in the paper's order:
  Eq. 25  D_ab = 1/2 sum_cij <ac||ij> <ij||bc> / (eps_ij^ac eps_ij^bc)
  Eq. 26  D V = V eta                (natural spinors, occupation numbers)
  Eq. 27  V~ = V T, keep eta_i >= eta_crit
  Eq. 28  F~ = V~^H F V~             (F = diag(eps_vir), canonical reference)
  Eq. 29  F~ Z~ = Z~ eps~            (semicanonicalisation)
  Eq. 30  U = V~ Z~                  (the paper calls this matrix B)
and the Cholesky vectors in the truncated basis: B'_vv = U^H B_vv U,
B'_ov = B_ov U, B'_vo = U^H B_vo, B'_oo = B_oo (the MO transformation of
Eq. 42 applied to the virtual block).
With ``t_ij^ab = <ab||ij>/eps_ij^ab`` Eq. 25 reads D_ab = 1/2 sum t_ij^ac conj(t_ij^bc).
"""
from __future__ import annotations

import numpy as np

from .integrals import eri

__all__ = ["fns_density", "fns_basis", "transform_cholesky"]


def fns_density(B, eps_occ, eps_vir):
    """Eq. 25, literally: numerator <ac||ij><ij||bc>, denominators eps_ij^ac eps_ij^bc."""
    eo = np.asarray(eps_occ, np.float64)
    ev = np.asarray(eps_vir, np.float64)
    o = eo.shape[0]
    vvoo = eri(B, o, "vvoo")  # <ac||ij> [a, c, i, j]
    oovv = eri(B, o, "oovv")  # <ij||bc> [i, j, b, c]
    den = (eo[None, None, :, None] + eo[None, None, None, :]
           - ev[:, None, None, None] - ev[None, :, None, None])  # eps_ij^ac  [a, c, i, j]
    ta = vvoo / den
    tb = oovv / den.transpose(2, 3, 0, 1)  # [i, j, b, c] / eps_ij^bc
    return 0.5 * np.einsum("acij,ijbc->ab", ta, tb)


def fns_basis(D, eps_vir, eta_crit):
    """Eqs. 26-30. Returns (eta descending, V, n_keep, U = V~ Z~, eps~ ascending)."""
    ev = np.asarray(eps_vir, np.float64)
    H = 0.5 * (D + D.conj().T)
    w, V = np.linalg.eigh(H)
    order = np.argsort(-w, kind="stable")
    eta, V = w[order], V[:, order]
    keep = eta >= eta_crit
    n_keep = int(np.count_nonzero(keep))
    Vt = V[:, keep]
    Ft = Vt.conj().T @ np.diag(ev) @ Vt
    et, Zt = np.linalg.eigh(0.5 * (Ft + Ft.conj().T))
    U = Vt @ Zt
    return eta, V, n_keep, U, et


def transform_cholesky(B, nocc, U):
    """Cholesky vectors in the occupied + truncated-virtual basis."""
    o = nocc
    nk = U.shape[1]
    Bn = np.empty((B.shape[0], o + nk, o + nk), dtype=np.complex128)
    Bn[:, :o, :o] = B[:, :o, :o]
    Bn[:, :o, o:] = B[:, :o, o:] @ U
    Bn[:, o:, :o] = U.conj().T @ B[:, o:, :o]
    Bn[:, o:, o:] = U.conj().T @ B[:, o:, o:] @ U
    return Bn
