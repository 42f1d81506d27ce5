"""Dense and Davidson eigensolvers for the lowest roots of M (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The secular problem is ``M X = X Omega`` with ``X^H X = 1`` (Eq. 10). "Lowest
roots" are the algebraically smallest eigenvalues of M.
"""
from __future__ import annotations

import numpy as np

__all__ = ["lowest_dense", "davidson"]


def lowest_dense(M, k):
    """Lowest k eigenpairs of a Hermitian matrix by LAPACK (numpy eigh)."""
    H = 0.5 * (M + M.conj().T)
    w, V = np.linalg.eigh(H)
    return w[:k], V[:, :k]


def davidson(sigma, diag, n, nroots, tol=1e-8, max_iter=200, max_space=None, guess=None):
    """Plain block Davidson (FP64) for the lowest ``nroots`` eigenpairs.

    ``sigma(V)`` maps a ``[k][n]`` block to ``M V``; ``diag`` is the exact
    diagonal of M (the preconditioner ``(omega - diag)^-1``). Convergence:
    every root's residual 2-norm ``||M y - omega y|| <= tol``.
    Returns (omega, Y[nroots][n], residual_norms, iterations).
    """
    diag = np.asarray(diag, dtype=np.float64)
    nguess = min(n, max(2 * nroots, nroots + 4))
    max_space = max_space or min(n, max(8 * nroots, 40))
    if guess is None:
        idx = np.argsort(diag, kind="stable")[:nguess]
        V = np.zeros((nguess, n), dtype=np.complex128)
        V[np.arange(nguess), idx] = 1.0
    else:
        V = np.array(guess, dtype=np.complex128)
        V, _ = np.linalg.qr(V.T)
        V = V.T
    S = sigma(V)
    for it in range(1, max_iter + 1):
        G = V.conj() @ S.T
        G = 0.5 * (G + G.conj().T)
        w, c = np.linalg.eigh(G)
        w, c = w[:nroots], c[:, :nroots]
        Y = c.T @ V
        SY = c.T @ S
        R = SY - w[:, None] * Y
        rn = np.linalg.norm(R, axis=1)
        if np.all(rn <= tol):
            return w, Y, rn, it
        if V.shape[0] + nroots > max_space:
            V, S = Y.copy(), SY.copy()
            # re-orthonormalise the collapsed space
            q, r = np.linalg.qr(V.T)
            V = q.T
            S = np.linalg.inv(r).T @ S
        new = []
        for r_, w_, rn_ in zip(R, w, rn):
            if rn_ <= tol:
                continue
            den = w_ - diag
            den = np.where(np.abs(den) < 1e-8, 1e-8, den)
            new.append(r_ / den)
        T = np.array(new)
        for _ in range(2):
            T = T - (T @ V.conj().T) @ V
        keep = []
        for t in T:
            for q in keep:
                t = t - np.vdot(q, t) * q
            nt = np.linalg.norm(t)
            if nt > 1e-10:
                keep.append(t / nt)
        if not keep:
            return w, Y, rn, it
        T = np.array(keep)
        V = np.concatenate([V, T])
        S = np.concatenate([S, sigma(T)])
    return w, Y, rn, max_iter
