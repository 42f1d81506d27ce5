"""Brute-force intermediate-state representation in determinant space.

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

This is the pin of the closed-form ADC blocks. For tiny spinor spaces it
builds the second-quantised Hamiltonian exactly in Fock space and follows the
construction of the ISR literally (Sec. 2.1):

* the correlated ground state ``Psi_0`` is expanded by Rayleigh-Schroedinger
  perturbation theory as a truncated power series in the coupling ``lam``,
  with ``H(lam) = H0 + lam*V`` where ``H0 = sum_p eps_p a+_p a_p`` and ``V``
  is the fluctuation potential, so that the Fock operator stays
  ``diag(eps)`` and the reference determinant stays the Hartree-Fock one for
  every ``lam``;
* the correlated excited states ``C_J Psi_0`` (Eq. 1) with the operator
  manifolds of Eqs. 2-4 (EE ``a+_a a_i``, ``a+_a a_i a+_b a_j``; IP ``a_i``,
  ``a+_a a_i a_j``; EA ``a+_a``, ``a+_a a+_b a_j``) are Gram-Schmidt
  orthogonalised against the already orthonormal lower classes (Eq. 5) and
  then symmetrically orthonormalised within each class (Eq. 6);
* the secular matrix ``M_IJ = <Psi~_I|H - E_0|Psi~_J>`` (Eq. 7) is formed,
  every product taken in truncated power-series arithmetic, so the returned
  Taylor coefficients are the perturbation orders ``M^(n)`` of Eq. 11
  exactly (up to rounding).

It also gives exact (FCI) energies in the N, N-1 and N+1 electron sectors for
the order-of-error test, and the brute-force MP1 one-particle density for the
natural-spinor pin.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np
import scipy.sparse as sp

__all__ = ["FockSpace", "antisym_eri_dense", "rspt_ground_state", "isr_series",
           "class_indices", "fci_energies", "mp1_density_bruteforce", "transition_moments_series",
           "spectroscopic_series"]


def antisym_eri_dense(B):
    """<pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr)  (Eq. 43), full dense array."""
    J = np.einsum("Qpr,Qqs->pqrs", B, B)
    return J - J.transpose(0, 1, 3, 2)


class FockSpace:
    """Determinants of ``nel`` electrons in ``nmo`` spinors as sorted tuples.

    A determinant ``(d0 < d1 < ...)`` stands for ``a+_{d0} a+_{d1} ... |vac>``.
    """

    def __init__(self, nmo):
        self.nmo = nmo
        self._dets = {}
        self._index = {}
        self._ann = {}

    def dets(self, nel):
        if nel not in self._dets:
            d = list(itertools.combinations(range(self.nmo), nel))
            self._dets[nel] = d
            self._index[nel] = {t: i for i, t in enumerate(d)}
        return self._dets[nel]

    def dim(self, nel):
        return comb(self.nmo, nel)

    def ann(self, p, nel):
        """Matrix of a_p from the nel-electron sector to the nel-1 sector."""
        key = (p, nel)
        if key not in self._ann:
            src = self.dets(nel)
            self.dets(nel - 1)
            idx = self._index[nel - 1]
            rows, cols, vals = [], [], []
            for c, d in enumerate(src):
                if p in d:
                    pos = d.index(p)
                    new = d[:pos] + d[pos + 1:]
                    rows.append(idx[new])
                    cols.append(c)
                    vals.append(-1.0 if pos % 2 else 1.0)
            self._ann[key] = sp.csr_matrix((vals, (rows, cols)),
                                           shape=(self.dim(nel - 1), self.dim(nel)))
        return self._ann[key]

    def cre(self, p, nel):
        """Matrix of a+_p from the nel-electron sector to the nel+1 sector."""
        return self.ann(p, nel + 1).T.tocsr()

    def excitation(self, p, q, nel):
        """E_pq = a+_p a_q within the nel-electron sector."""
        return (self.cre(p, nel - 1) @ self.ann(q, nel)).tocsr()

    def det_index(self, nel, det):
        self.dets(nel)
        return self._index[nel][tuple(det)]


def _hamiltonian_parts(fs, eps, g, nel):
    """H0 and the fluctuation potential V in the nel sector (complex sparse).

    H0 = sum_p eps_p E_pp.
    V  = 1/4 sum <pq||rs> a+p a+q a_s a_r - sum_pq u_pq E_pq,
    u_pq = sum_k <pk||qk> over the occupied k of the reference, so that the
    full one-particle operator is h = diag(eps) - lam*u and the Fock matrix
    stays diag(eps) for every coupling strength.
    """
    nmo = fs.nmo
    nocc = fs._nocc
    dim = fs.dim(nel)
    E = [[fs.excitation(p, q, nel).tocoo() for q in range(nmo)] for p in range(nmo)]
    h0 = np.zeros(dim)
    for p in range(nmo):
        h0 += eps[p] * E[p][p].tocsr().diagonal()
    u = np.einsum("pkqk->pq", g[:, :nocc, :, :nocc])
    # stacked coordinates of every E_qs, tagged with its (q, s) id
    rows = np.concatenate([E[q][s].row for q in range(nmo) for s in range(nmo)])
    cols = np.concatenate([E[q][s].col for q in range(nmo) for s in range(nmo)])
    vals = np.concatenate([E[q][s].data for q in range(nmo) for s in range(nmo)])
    tag = np.concatenate([np.full(E[q][s].nnz, q * nmo + s) for q in range(nmo) for s in range(nmo)])
    V = sp.csr_matrix((dim, dim), dtype=np.complex128)
    # 1/4 sum g_pqrs a+p a+q a_s a_r, with a+p a+q a_s a_r = E_pr E_qs - delta_qr E_ps
    for p in range(nmo):
        for r in range(nmo):
            coef = g[p, :, r, :].ravel()[tag]
            W = sp.csr_matrix((coef * vals, (rows, cols)), shape=(dim, dim))
            V = V + 0.25 * (E[p][r].tocsr() @ W)
    for p in range(nmo):
        for s in range(nmo):
            c = 0.25 * np.trace(g[p, :, :, s]) + u[p, s]
            if c != 0.0:
                V = V - c * E[p][s].tocsr()
    return h0, V.tocsr()


class _Sector:
    def __init__(self, fs, eps, g, nel):
        self.nel = nel
        self.h0, self.V = _hamiltonian_parts(fs, eps, g, nel)
        self.dim = self.h0.shape[0]

    def H(self, lam):
        return sp.diags(self.h0).tocsr() + lam * self.V


def _build_space(eps, g, nocc):
    nmo = eps.shape[0]
    fs = FockSpace(nmo)
    fs._nocc = nocc
    return fs


# ---------------------------------------------------------------------------
# truncated power-series arithmetic: a series is an array whose first axis is
# the perturbation order
# ---------------------------------------------------------------------------

def _sdot(A, B):
    """<A|B> for state series A[n, a, dim], B[n, b, dim] -> [n, a, b]."""
    nord = A.shape[0]
    out = np.zeros((nord, A.shape[1], B.shape[1]), dtype=np.complex128)
    for n in range(nord):
        for m in range(n + 1):
            out[n] += A[m].conj() @ B[n - m].T
    return out


def _smat(X, Y):
    """Matrix series product X[n, a, b] @ Y[n, b, c]."""
    nord = X.shape[0]
    out = np.zeros((nord, X.shape[1], Y.shape[2]), dtype=np.complex128)
    for n in range(nord):
        for m in range(n + 1):
            out[n] += X[m] @ Y[n - m]
    return out


def _scombine(S, C):
    """States S[n, k, dim] combined with coefficients C[n, k, j]: sum_k S_k C_kj."""
    nord = S.shape[0]
    out = np.zeros((nord, C.shape[2], S.shape[2]), dtype=np.complex128)
    for n in range(nord):
        for m in range(n + 1):
            out[n] += C[n - m].T @ S[m]
    return out


def _inv_sqrt(S):
    """(I + X)^(-1/2) for a Hermitian series S with S^(0) = I, by the binomial series."""
    nord, k, _ = S.shape
    if not np.allclose(S[0], np.eye(k), atol=1e-12):
        raise ValueError("zeroth-order overlap is not the identity")
    X = S.copy()
    X[0] = 0.0
    out = np.zeros_like(S)
    out[0] = np.eye(k)
    P = np.zeros_like(S)
    P[0] = np.eye(k)
    coef = 1.0
    for j in range(1, nord):
        coef *= (-0.5 - (j - 1)) / j
        P = _smat(P, X)
        out += coef * P
    return out


def rspt_ground_state(sector, phi_index, nord):
    """Rayleigh-Schroedinger series of the ground state (intermediate normalisation).

    Returns (Psi[n, dim], E[n]) with H = H0 + lam V.
    """
    dim = sector.dim
    E0 = sector.h0[phi_index]
    denom = E0 - sector.h0
    denom[phi_index] = np.inf
    R0 = 1.0 / denom
    R0[phi_index] = 0.0
    psi = np.zeros((nord, dim), dtype=np.complex128)
    psi[0, phi_index] = 1.0
    E = np.zeros(nord, dtype=np.complex128)
    E[0] = E0
    for n in range(1, nord):
        E[n] = (sector.V @ psi[n - 1])[phi_index]
        rhs = sector.V @ psi[n - 1]
        for k in range(1, n + 1):
            rhs = rhs - E[k] * psi[n - k]
        psi[n] = R0 * rhs
    return psi, E


def class_indices(kind, nocc, nvir):
    """Labels of the ISR classes, in the packed order used everywhere.

    IP: 1h ``i``; 2h1p ``(i<j, a)`` with ``a`` fastest, operator ``a+_a a_i a_j``.
    EA: 1p ``a``; 2p1h ``(j, a<b)`` with the pair fastest, operator ``a+_a a+_b a_j``.
    EE: 1h1p ``(i, a)``, operator ``a+_a a_i``; 2h2p ``(i<j, a<b)``,
        operator ``a+_a a_i a+_b a_j``.
    Orbital numbers are absolute (virtual ``a`` is ``nocc + a``).
    """
    o, v = nocc, nvir
    occ = list(range(o))
    vir = list(range(o, o + v))
    opairs = [(i, j) for i in occ for j in occ if i < j]
    vpairs = [(a, b) for a in vir for b in vir if a < b]
    if kind == "IP":
        return [[(i,) for i in occ], [(i, j, a) for (i, j) in opairs for a in vir]]
    if kind == "EA":
        return [[(a,) for a in vir], [(j, a, b) for j in occ for (a, b) in vpairs]]
    if kind == "EE":
        return [[(i, a) for i in occ for a in vir],
                [(i, j, a, b) for (i, j) in opairs for (a, b) in vpairs]]
    raise ValueError(kind)


def _class_operator(fs, kind, cls, label, nel):
    """Matrix of C_J from the N sector to the target sector."""
    if kind == "IP":
        if cls == 0:
            (i,) = label
            return fs.ann(i, nel)
        i, j, a = label
        return fs.cre(a, nel - 2) @ fs.ann(i, nel - 1) @ fs.ann(j, nel)
    if kind == "EA":
        if cls == 0:
            (a,) = label
            return fs.cre(a, nel)
        j, a, b = label
        return fs.cre(a, nel) @ fs.cre(b, nel - 1) @ fs.ann(j, nel)
    if kind == "EE":
        if cls == 0:
            i, a = label
            return fs.excitation(a, i, nel)
        i, j, a, b = label
        return fs.excitation(a, i, nel) @ fs.excitation(b, j, nel)
    raise ValueError(kind)


def isr_series(eps, B, nocc, kind, nord=4, want_states=False):
    """Exact perturbation orders of the ISR secular matrix for a tiny case.

    With want_states the intermediate states themselves are returned instead
    (``states`` [nord, N, dim] in the target sector, and for EE the
    normalised ground-state series ``psi0`` [nord, dim]).

    Returns dict with
      ``M``: [nord, N, N] series (class 1 states first, then class 2),
      ``n1``: number of class-1 states,
      ``E``: ground-state energy series,
      ``labels``: class labels (see class_indices).
    """
    eps = np.asarray(eps, dtype=np.float64)
    nmo = eps.shape[0]
    nvir = nmo - nocc
    g = antisym_eri_dense(B)
    fs = _build_space(eps, g, nocc)
    secN = _Sector(fs, eps, g, nocc)
    phi = fs.det_index(nocc, tuple(range(nocc)))
    psi, E = rspt_ground_state(secN, phi, nord)
    if kind == "IP":
        tgt = nocc - 1
    elif kind == "EA":
        tgt = nocc + 1
    else:
        tgt = nocc
    sec_t = secN if tgt == nocc else _Sector(fs, eps, g, tgt)
    classes = class_indices(kind, nocc, nvir)

    ortho = []  # list of [nord, k, dim] orthonormal class series
    if kind == "EE":
        nrm = _sdot(psi[:, None, :], psi[:, None, :])
        inv = _inv_sqrt(nrm)
        ortho.append(_scombine(psi[:, None, :], inv))
    excited = []
    for cls, labels in enumerate(classes):
        ops = [_class_operator(fs, kind, cls, lab, nocc) for lab in labels]
        ces = np.zeros((nord, len(labels), sec_t.dim), dtype=np.complex128)
        for n in range(nord):
            for k, op in enumerate(ops):
                ces[n, k] = op @ psi[n]
        prec = ces.copy()
        for low in ortho:
            ov = _sdot(low, ces)
            prec = prec - _scombine(low, ov)
        S = _sdot(prec, prec)
        tilde = _scombine(prec, _inv_sqrt(S))
        ortho.append(tilde)
        excited.append(tilde)
    states = np.concatenate(excited, axis=1)
    if want_states:
        return {"states": states, "psi0": ortho[0][:, 0, :] if kind == "EE" else None, "fs": fs,
                "nel": tgt, "n1": len(classes[0]), "labels": classes}
    # (H - E0) applied to the state series
    h0 = sec_t.h0
    HS = np.zeros_like(states)
    for n in range(nord):
        HS[n] += (h0[None, :] - E[0]) * states[n]
        if n >= 1:
            HS[n] += (sec_t.V @ states[n - 1].T).T - E[1] * states[n - 1]
        for k in range(2, n + 1):
            HS[n] -= E[k] * states[n - k]
    M = _sdot(states, HS)
    return {"M": M, "n1": len(classes[0]), "E": E, "labels": classes}


def fci_energies(eps, B, nocc, lam, nel, nroots=1):
    """Lowest exact eigenvalues of H(lam) in the nel-electron sector.

    H(lam) = sum_p eps_p E_pp + lam * V (Fock matrix diag(eps) for every lam).
    """
    eps = np.asarray(eps, dtype=np.float64)
    g = antisym_eri_dense(B)
    fs = _build_space(eps, g, nocc)
    sec = _Sector(fs, eps, g, nel)
    H = sec.H(lam).toarray()
    w = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
    return w[:nroots]


def mp1_density_bruteforce(eps, B, nocc):
    """rho_pq = <Psi1|a+_p a_q|Psi1> from the exact first-order wavefunction."""
    eps = np.asarray(eps, dtype=np.float64)
    nmo = eps.shape[0]
    g = antisym_eri_dense(B)
    fs = _build_space(eps, g, nocc)
    sec = _Sector(fs, eps, g, nocc)
    phi = fs.det_index(nocc, tuple(range(nocc)))
    psi, _ = rspt_ground_state(sec, phi, 2)
    p1 = psi[1]
    rho = np.zeros((nmo, nmo), dtype=np.complex128)
    for p in range(nmo):
        for q in range(nmo):
            rho[p, q] = np.vdot(p1, fs.excitation(p, q, nocc) @ p1)
    return rho, psi


def transition_moments_series(eps, B, nocc, nord=3):
    """EE transition moments f_I(pq) = <Psi~_I| a+_p a_q |Psi0> as a series.

    Intermediate states of the ISR (Eqs. 5-6, as in isr_series) and the
    normalised ground state, both as perturbation series; returns
    f [nord, N, nmo, nmo] (class 1 first, labels as class_indices).
    """
    r = isr_series(eps, B, nocc, "EE", nord=nord, want_states=True)
    fs, nel, states, psi0 = r["fs"], r["nel"], r["states"], r["psi0"]
    nmo = fs.nmo
    N = states.shape[1]
    f = np.zeros((nord, N, nmo, nmo), dtype=np.complex128)
    for p in range(nmo):
        for q in range(nmo):
            E = fs.excitation(p, q, nel)
            Epsi = np.stack([E @ psi0[n] for n in range(nord)])  # [nord, dim]
            f[:, :, p, q] = _sdot(states, Epsi[:, None, :])[:, :, 0]
    return f, r["n1"], r["labels"]


def spectroscopic_series(eps, B, nocc, kind, nord=3):
    """IP/EA transition moments f_I(p) = <Psi~_I| a_p |Psi0> (IP) or <Psi~_I| a+_p |Psi0> (EA).

    Intermediate states of the (N-1)/(N+1) ISR (as in isr_series) and the
    normalised N-electron ground state, both perturbation series; returns
    f [nord, N, nmo] (class 1 first, labels as class_indices).
    """
    eps = np.asarray(eps, dtype=np.float64)
    r = isr_series(eps, B, nocc, kind, nord=nord, want_states=True)
    fs, nel, states = r["fs"], r["nel"], r["states"]
    g = antisym_eri_dense(B)
    secN = _Sector(fs, eps, g, nocc)
    phi = fs.det_index(nocc, tuple(range(nocc)))
    psi, _ = rspt_ground_state(secN, phi, nord)
    nrm = _sdot(psi[:, None, :], psi[:, None, :])
    psi0 = _scombine(psi[:, None, :], _inv_sqrt(nrm))[:, 0, :]
    nmo = fs.nmo
    f = np.zeros((nord, states.shape[1], nmo), dtype=np.complex128)
    for p in range(nmo):
        op = fs.ann(p, nocc) if kind == "IP" else fs.cre(p, nocc)
        ops = np.stack([op @ psi0[n] for n in range(nord)])
        f[:, :, p] = _sdot(states, ops[:, None, :])[:, :, 0]
    return f, r["n1"], r["labels"]

