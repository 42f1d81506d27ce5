"""One-step pivoted Cholesky decomposition of the two-electron integrals and
the transformation of the vectors to molecular spinors (oracle), Sec. 2.5.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. 41: (mu nu|kappa lambda) ~ sum_P L^P_(mu nu) L^P_(kappa lambda). The
vectors are generated one at a time from the positive semidefinite matrix
V[(mu nu)][(kappa lambda)]: take the largest remaining diagonal element
d_max (stop when d_max < tau), then
    L^P = (V[:, piv] - sum_{P' < P} L^P' L^P'_piv) / sqrt(d_max),
    d <- d - (L^P)^2.
Every residual diagonal then lies below tau, and since the residual matrix is
positive semidefinite every residual element is bounded by tau as well.
Eq. 42: L^P_pq = sum_(mu nu) conj(C_mu p) L^P_(mu nu) C_nu q (the B of the ADC
input); with real L symmetric in (mu nu) each B^P is Hermitian.
"""
from __future__ import annotations

import numpy as np

__all__ = ["pivoted_cholesky", "to_mo"]


def pivoted_cholesky(V, tau, max_rank=None):
    """(L [rank][n], pivots) of the PSD matrix V [n][n] down to diagonal tau."""
    V = np.asarray(V, np.float64)
    n = V.shape[0]
    max_rank = n if max_rank is None else int(max_rank)
    d = np.diag(V).copy()
    L = np.zeros((max_rank, n))
    piv = []
    for P in range(max_rank):
        j = int(np.argmax(d))
        dmax = d[j]
        if not dmax >= tau or dmax <= 0.0:
            break
        col = V[:, j] - L[:P].T @ L[:P, j]
        L[P] = col / np.sqrt(dmax)
        d = d - L[P] ** 2
        d[j] = 0.0
        piv.append(j)
    r = len(piv)
    return L[:r].copy(), np.array(piv, dtype=np.int64)


def to_mo(L, nao, C):
    """B[P] = C^H L^P C for L [rank][nao*nao] and C [nao][nmo] (Eq. 42)."""
    Lm = np.asarray(L).reshape(-1, nao, nao)
    return np.einsum("mp,Pmn,nq->Ppq", C.conj(), Lm, C)
