"""The small Hermitian eigensolvers of the Davidson's Rayleigh-Ritz step (Eq. 10
projected onto the subspace) against LAPACK (numpy.linalg.eigh): FP64 Jacobi
and the FP32 Jacobi start refined in FP64, on random Hermitian matrices with
the spectra the Davidson meets (a large common shift, spread of a few hundred),
including exactly degenerate pairs (time-reversal doubling) and pairs closer
than FP32 can resolve. Eigenvalues within 1e-13 of the spectral norm,
residuals ||A v - w v|| within 1e-13 of it, eigenvectors orthonormal to 1e-13;
eigenvectors of degenerate pairs are not unique, so only these properties are
compared. The spectra with clusters take the refinement through its coupled
clusters (exact diagonalisation of each), through clusters that split as the
vectors improve, and (ten-fold) to its FP64 Jacobi fallback. The refined solver is for matrices whose eigenvalues
are needed to absolute accuracy (the Rayleigh-Ritz step); small eigenvalues of
a positive definite matrix keep only absolute accuracy there, which is why the
Davidson's Gram matrices of new directions stay with the FP64 Jacobi."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _hermitian(n, seed, spectrum=None, shift=-3700.0, spread=300.0):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    U, _ = np.linalg.qr(Z)
    lam = shift + spread * np.sort(rng.uniform(-1.0, 1.0, n)) if spectrum is None else np.asarray(spectrum, float)
    A = (U * lam) @ U.conj().T
    return 0.5 * (A + A.conj().T)


def _check(A, w, V, orth=1e-13):
    nrm = np.abs(np.linalg.eigvalsh(A)).max()
    wr = np.linalg.eigvalsh(A)
    assert np.abs(w - wr).max() < 1e-13 * nrm, np.abs(w - wr).max() / nrm
    res = np.linalg.norm(A @ V - V * w, axis=0).max()
    assert res < 1e-13 * nrm, res / nrm
    assert np.abs(V.conj().T @ V - np.eye(A.shape[0])).max() < orth


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 8, 17, 33, 64, 100, 128])
def test_eigh_random(gpu, which, n):
    A = _hermitian(n, seed=70 + n)
    w, V, ms, steps = gpu.diag_eigh(which, A)
    _check(A, w, V)
    if which == 1:
        assert steps >= 3, steps   # refined, no fallback on spectra without wide clusters


def _spectra():
    rng = np.random.default_rng(81)
    base = -3700.0 + 300.0 * np.sort(rng.uniform(-1.0, 1.0, 24))
    yield "pairs", np.concatenate([base, base, base[:8] + 1e-9, base[8:16] + 1e-6]), 82   # exact and near pairs
    # converging Davidson roots: two near pairs below a spread of higher Ritz values
    yield "ritz", np.concatenate([[0.8382872629, 0.8382872629 + 1e-12, 0.898, 0.898 + 1e-11],
                                  np.sort(np.random.default_rng(5).uniform(0.9, 5.0, 28))]), 3
    # six eigenvalues 1e-7 apart: one cluster at first, separate pairs later
    yield "six", np.concatenate([1.0 + 1e-7 * np.arange(6), np.linspace(2.0, 3.0, 20)]), 5
    # time-reversal pairs split by 1e-13
    yield "kramers", np.repeat(np.linspace(-5.0, 5.0, 16), 2) + np.tile([0.0, 1e-13], 16), 6
    # a ten-fold eigenvalue: wider than the refinement's exact cluster step (FP64 Jacobi instead)
    yield "tenfold", np.concatenate([np.full(10, 1.0), np.linspace(2.0, 3.0, 20)]), 4


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("case", ["pairs", "ritz", "six", "kramers", "tenfold"])
def test_eigh_degenerate_and_close(gpu, which, case):
    _, lam, seed = next(c for c in _spectra() if c[0] == case)
    A = _hermitian(lam.size, seed=seed, spectrum=lam)
    w, V, ms, steps = gpu.diag_eigh(which, A)
    _check(A, w, V)
    if which == 1:
        # only the ten-fold eigenvalue needs the FP64 Jacobi
        assert (steps == -1) == (case == "tenfold"), steps


def test_eigh_refined_is_faster(gpu):
    """At the Davidson's usual subspace size the refined solver beats the FP64 Jacobi."""
    A = _hermitian(64, seed=90)
    # best of three calls each, so that one-time costs (module loading) and a
    # busy moment on the device do not decide the comparison
    t0 = min(gpu.diag_eigh(0, A)[2] for _ in range(3))
    t1 = min(gpu.diag_eigh(1, A)[2] for _ in range(3))
    print(f"n = 64: FP64 Jacobi {t0:.3f} ms, FP32 start + FP64 refinement {t1:.3f} ms")
    assert t1 < t0
