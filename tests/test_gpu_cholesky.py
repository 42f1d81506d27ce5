"""Pivoted Cholesky decomposition and MO transformation on the GPU
(adc_cholesky, adc_cholesky_mo; Sec. 2.5, Eqs. 41-42) against the oracle:
the same rank and pivots on generic inputs (distinct diagonals), the vectors to
1e-12 relative, every residual element below tau, the spinor-basis vectors to
1e-13, and an ADC context built from them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_eri, random_unitary  # noqa: E402
from oracle.cholesky import pivoted_cholesky, to_mo  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


@pytest.mark.parametrize("nao,rank,tau,seed", [(8, 30, 1e-8, 81), (6, 20, 1e-4, 82), (10, 45, 1e-6, 83)])
def test_cholesky_matches_oracle(gpu, nao, rank, tau, seed):
    V = make_eri(nao, rank, seed=seed, decay=0.7)
    L, piv = gpu.cholesky(V, tau)
    Lr, pr = pivoted_cholesky(V, tau)
    assert L.shape == Lr.shape and np.array_equal(piv, pr)
    assert np.abs(L - Lr).max() < 1e-12 * np.abs(Lr).max()
    R = V - L.T @ L
    assert np.abs(R).max() < tau * (1 + 1e-9)


def test_cholesky_full_rank_and_mo(gpu):
    rng = np.random.default_rng(84)
    nao = 6
    A = rng.standard_normal((nao * nao, nao * nao))
    V = A @ A.T + np.eye(nao * nao)
    L, piv = gpu.cholesky(V, 0.0)
    Lr, pr = pivoted_cholesky(V, 0.0)
    assert L.shape[0] == nao * nao and np.array_equal(piv, pr)
    assert np.abs(L - Lr).max() < 1e-12 * np.abs(Lr).max()
    C = random_unitary(nao, seed=85)
    B = gpu.cholesky_mo(L, nao, C)
    Br = to_mo(Lr, nao, C)
    assert np.abs(B - Br).max() < 1e-13 * np.abs(Br).max()


def test_context_from_cholesky_vectors(gpu):
    nao, o = 7, 3
    V = make_eri(nao, 25, seed=86, decay=0.5)
    L, _ = gpu.cholesky(V, 1e-10)
    # symmetrise the AO vectors (Eq. 41 is symmetric in mu nu) and rotate to spinors
    Lm = L.reshape(-1, nao, nao)
    L = (0.5 * (Lm + Lm.transpose(0, 2, 1))).reshape(L.shape[0], -1)
    B = 0.05 * gpu.cholesky_mo(L, nao, random_unitary(nao, seed=87))
    eo = np.linspace(-2.0, -0.6, o)
    ev = np.linspace(0.3, 3.0, nao - o)
    with gpu.Context(B, eo, ev, kind="EA", order=2) as c:
        w, _, e64, _, rc = c.davidson(2, tol=1e-8, want_vectors=False)
    assert rc == 0 and np.all(np.isfinite(w))
