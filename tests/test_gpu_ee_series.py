"""The device's EE-ADC matrix against the brute-force ISR series directly.

The EE term tables of the library and those of the oracle are two
transcriptions of one derivation, and GPU-vs-oracle parity only shows that
the device evaluates its tables as the oracle evaluates its own. These tests
skip the closed forms altogether: the perturbation orders M^(0..3) of the
intermediate-state matrix come from the determinant-space construction of
Sec. 2.1 (correlated excited states, Gram-Schmidt against the lower classes,
symmetric orthonormalisation, M = <Psi~|H - E0|Psi~>, Eqs. 1, 5-7, 11), and the
device's singles block, its whole matrix (sigma of the unit vectors) and its
adjoint's x-derivative are compared with them (Eq. 12 with every ADC(3) term
scaled by x: singles M^(3), coupling M^(2), doubles M^(1))."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle.isr_series import isr_series  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _series_matrix(M, n1, order, x, dd):
    """ADC(2) or ADC(2)+x(3) from the series orders; dd = 0 keeps the doubles block at zeroth order."""
    xs = x if order == 3 else 0.0
    A = M[0] + M[1] + M[2]
    A[:n1, :n1] += xs * M[3][:n1, :n1]
    A[:n1, n1:] -= M[2][:n1, n1:]
    A[n1:, :n1] -= M[2][n1:, :n1]
    A[:n1, n1:] += xs * M[2][:n1, n1:]
    A[n1:, :n1] += xs * M[2][n1:, :n1]
    A[n1:, n1:] = M[0][n1:, n1:] + (xs * M[1][n1:, n1:] if dd == 1 else 0.0)
    return A


def _delta(M, n1, dd):
    """dM/dx: the terms ADC(3) adds to ADC(2)."""
    D = np.zeros_like(M[0])
    D[:n1, :n1] = M[3][:n1, :n1]
    D[:n1, n1:] = M[2][:n1, n1:]
    D[n1:, :n1] = M[2][n1:, :n1]
    if dd == 1:
        D[n1:, n1:] = M[1][n1:, n1:]
    return D


@pytest.mark.parametrize("o,v,Q,seed", [(3, 4, 6, 3), (2, 5, 6, 7), (4, 3, 6, 9)])
def test_ee_device_matrix_equals_isr_series(gpu, o, v, Q, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.3)
    r = isr_series(np.concatenate([p.eps_occ, p.eps_vir]), p.B, o, "EE", nord=4)
    M, n1 = r["M"], r["n1"]
    scale = max(1.0, np.abs(M[0]).max())
    for order, x, dd in ((3, 0.7, 1), (3, 1.0, 0), (2, 0.0, 1)):
        ref = _series_matrix(M, n1, order, x, dd)
        with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=order, x=x, dd_order=dd) as ctx:
            assert ctx.n1 == n1 and ctx.N == ref.shape[0]
            main = ctx.main_block()
            S = ctx.sigma(np.eye(ctx.N, dtype=np.complex128), "fp64")
        assert np.abs(main - ref[:n1, :n1]).max() < 1e-12 * scale, (order, x, dd, "singles block")
        assert np.abs(S.T - ref).max() < 1e-12 * scale, (order, x, dd, "matrix")


@pytest.mark.parametrize("o,v,Q,seed,dd", [(3, 4, 6, 3, 1), (2, 5, 6, 7, 0)])
def test_ee_adjoint_x_derivative_equals_isr_series(gpu, o, v, Q, seed, dd):
    """d/dx of sum_r g_r y_r^H M y_r = sum_r g_r y_r^H dM/dx y_r, M linear in x (Eq. 12)."""
    p = make_problem(o, v, Q, seed=seed, sigma=0.3)
    r = isr_series(np.concatenate([p.eps_occ, p.eps_vir]), p.B, o, "EE", nord=4)
    M, n1 = r["M"], r["n1"]
    D = _delta(M, n1, dd)
    g = np.array([1.0, -0.5, 0.25])
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=0.6, dd_order=dd) as ctx:
        Y = random_vectors(ctx.N, 3, seed=seed + 2)
        _, _, _, gx = ctx.sigma_adjoint(Y, g)
    ref = float(sum(gr * np.real(np.vdot(y, D @ y)) for gr, y in zip(g, Y)))
    assert abs(gx - ref) < 1e-11 * max(1.0, abs(ref)), (gx, ref)
