"""Pins of the pivoted Cholesky oracle (Sec. 2.5, Eqs. 41-42).

* An exactly low-rank PSD matrix is reproduced with exactly its rank.
* With a threshold tau every element of the residual V - L^T L lies below tau
  (the residual is PSD with diagonal below tau).
* On a positive definite matrix the vectors in pivot order are the transposed
  Cholesky factor of the pivoted matrix (numpy.linalg.cholesky).
* Eq. 42: every B^P is Hermitian, and sum_P B^P_pq B^P_rs equals the
  four-index transformation of the reconstructed AO integrals.
"""
import numpy as np
import pytest

from synthetic import make_eri, random_unitary
from oracle.cholesky import pivoted_cholesky, to_mo


@pytest.mark.parametrize("nao,rank,seed", [(5, 7, 1), (6, 12, 2), (4, 3, 3)])
def test_low_rank_is_exact(nao, rank, seed):
    V = make_eri(nao, rank, seed=seed)
    L, piv = pivoted_cholesky(V, 1e-12 * np.abs(V).max())
    assert L.shape[0] == rank
    assert np.abs(V - L.T @ L).max() < 1e-11 * np.abs(V).max()
    assert len(set(piv.tolist())) == len(piv)


@pytest.mark.parametrize("tau", [1e-2, 1e-4, 1e-6])
def test_threshold_bounds_every_element(tau):
    V = make_eri(7, 40, seed=4, decay=0.6)
    L, _ = pivoted_cholesky(V, tau)
    R = V - L.T @ L
    assert np.diag(R).max() < tau
    assert np.abs(R).max() < tau * (1 + 1e-9)
    assert L.shape[0] < 40


def test_positive_definite_matches_library_cholesky():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 30))
    V = A @ A.T + 30 * np.eye(30)
    L, piv = pivoted_cholesky(V, 0.0)
    assert L.shape[0] == 30
    K = np.linalg.cholesky(V[np.ix_(piv, piv)])  # lower triangular
    assert np.abs(L[:, piv] - K.T).max() < 1e-12 * np.abs(K).max()


def test_mo_transform():
    nao = 5
    V = make_eri(nao, 9, seed=6)
    L, _ = pivoted_cholesky(V, 1e-13)
    C = random_unitary(nao, seed=7)[:, :4]  # four molecular spinors
    B = to_mo(L, nao, C)
    assert np.abs(B - B.conj().transpose(0, 2, 1)).max() < 1e-13
    Vr = (L.T @ L).reshape(nao, nao, nao, nao)
    mo = np.einsum("mp,nq,kr,ls,mnkl->pqrs", C.conj(), C, C.conj(), C, Vr)
    assert np.abs(np.einsum("Ppq,Prs->pqrs", B, B) - mo).max() < 1e-12 * np.abs(mo).max()
