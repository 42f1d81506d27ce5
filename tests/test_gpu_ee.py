"""EE-ADC on the GPU against the CPU oracle: sigma (FP64 and BF16x3), diagonal,
singles block and lowest roots (Sec. 2.1, Eq. 2 manifold). Tolerances as in
test_gpu_parity: 1e-12 relative per FP64 sigma vector, 1e-4 for the
split-precision one, 1e-8 Eh for eigenvalues (also after the mixed-precision
Davidson's FP64 refinement)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle import adc_ee  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _rel(S, R):
    return np.linalg.norm(S - R, axis=-1) / np.linalg.norm(R, axis=-1)


@pytest.mark.parametrize("o,v,Q,order,x,dd,seed", [
    (4, 8, 12, 3, 1.0, 1, 1),
    (5, 11, 20, 3, 0.4, 1, 2),
    (3, 7, 9, 3, 1.0, 0, 3),
    (6, 9, 14, 2, 0.0, 1, 4),
    (2, 2, 5, 3, 1.0, 1, 5),   # one occupied pair, one virtual pair
])
def test_ee_sigma_diag_block(gpu, o, v, Q, order, x, dd, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=order, x=x, dd_order=dd) as ctx:
        n1, n2 = adc_ee.dims(o, v)
        assert (ctx.n1, ctx.n2) == (n1, n2)
        T = adc_ee.Tensors(p.B, p.eps_occ, p.eps_vir)
        X = random_vectors(ctx.N, 3, seed=seed + 10)
        ref = adc_ee.sigma_ref(order, x, p.B, p.eps_occ, p.eps_vir, X, dd_order=dd, T=T)
        S = ctx.sigma(X, "fp64")
        assert _rel(S, ref).max() < 1e-12
        d = ctx.diagonal()
        dref = adc_ee.diagonal_ref(order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd, T=T)
        assert np.abs(d - dref).max() < 1e-12 * max(1.0, np.abs(dref).max())
        M = adc_ee.explicit_matrix(order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd)
        assert np.abs(ctx.main_block() - M[:n1, :n1]).max() < 1e-12 * np.abs(M).max()
        Sm = ctx.sigma(X, "bf16x3")
        assert _rel(Sm, ref).max() < 1e-4
        Sm6 = ctx.sigma(X, "bf16x6")
        assert _rel(Sm6, ref).max() < 1e-4, _rel(Sm6, ref).max()
        Ss = ctx.sigma(X, "sliced")
        assert _rel(Ss, ref).max() < 1e-10, _rel(Ss, ref).max()
        # the intermediate step: digits for about 24 bits
        Ss24 = ctx.sigma(X, "sliced24")
        assert _rel(Ss24, ref).max() < 2e-6, _rel(Ss24, ref).max()


@pytest.mark.parametrize("o,v,Q,x,dd,seed", [(4, 10, 14, 1.0, 0, 31), (3, 7, 11, 0.6, 1, 32)])
def test_ee_singles_block_chunked_four_virtual(gpu, o, v, Q, x, dd, seed):
    """Third-order singles block with its four-virtual rows in chunks of the
    first virtual index (v = 10: chunks 3, 3, 3, 1; v = 7: 2, 2, 2, 1), through
    the ladder intermediate and the Cholesky vectors instead of the dense
    <ab||cd>: equal to the oracle's explicit block and to the dense evaluation."""
    p = make_problem(o, v, Q, seed=seed, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    n1 = o * v
    M = adc_ee.explicit_matrix(3, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd)
    X = random_vectors(n1 + adc_ee.dims(o, v)[1], 2, seed=seed + 1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=x, dd_order=dd, vvvv="chunked") as c:
        Mc = c.main_block()
        Sc = c.sigma(X, "fp64")
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=x, dd_order=dd, vvvv="dense") as c:
        Md = c.main_block()
    assert np.abs(Mc - M[:n1, :n1]).max() < 1e-12 * np.abs(M).max()
    assert np.abs(Mc - Md).max() < 1e-13 * np.abs(Md).max()
    ref = adc_ee.sigma_ref(3, x, p.B, p.eps_occ, p.eps_vir, X, dd_order=dd)
    assert _rel(Sc, ref).max() < 1e-12


def test_ee_davidson_matches_dense(gpu):
    o, v, Q = 4, 9, 16
    p = make_problem(o, v, Q, seed=7, sigma=0.08, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    M = adc_ee.explicit_matrix(3, 0.4, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:4]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=0.4) as ctx:
        om, Y, e64, st, rc = ctx.davidson(4, tol=1e-8, precision="fp64")
    assert rc == 0
    assert np.abs(om - w).max() < 1e-8
    assert np.linalg.norm(Y @ M.T - om[:, None] * Y, axis=1).max() < 1e-7


@pytest.mark.parametrize("prec,refine", [("bf16x3", "fp64"), ("bf16x6", "fp64"), ("bf16x3", "sliced")])
def test_ee_mixed_davidson_refined(gpu, prec, refine):
    o, v, Q = 4, 10, 16
    p = make_problem(o, v, Q, seed=9, sigma=0.08, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    M = adc_ee.explicit_matrix(3, 0.4, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:4]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=0.4, refine=refine) as ctx:
        om, _, e64, st, rc = ctx.davidson(4, tol=1e-8, precision=prec, want_vectors=False)
    assert rc == 0 and np.all(e64 <= 1e-8)
    assert np.abs(om - w).max() < 1e-8
    assert st["sigma_calls_fp64"] < st["sigma_calls"]
