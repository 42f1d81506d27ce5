"""adc_sigma_share on one GPU: the shares of an EA problem split by the
satellites' occupied index, computed one rank after another on the same
device (no rank waits on another), assemble into the whole sigma: the sum of
the partial 1p rows and the concatenated satellite rows equal adc_sigma's
FP64 product and the oracle's term-by-term sigma (Sec. 2.1, Eqs. 10-12) to
1e-12, for ranges of one occupied index, uneven ranges and empty ones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle import adc as oadc  # noqa: E402


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


@pytest.mark.parametrize("order,x", [(3, 0.5), (3, 1.0), (2, 0.0)])
@pytest.mark.parametrize("world", [1, 2, 3, 7, 9])
def test_shares_assemble_into_sigma(gpu, order, x, world):
    from paper_2511_21640_gb300.shard import occupied_ranges
    o, v, Q = 7, 12, 20
    p = make_problem(o, v, Q, seed=64, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=order, x=x) as ctx:
        X = random_vectors(ctx.N, 3, seed=65)
        full = ctx.sigma(X, "fp64")
        n1 = ctx.n1
        main = np.zeros((3, n1), np.complex128)
        sats = []
        for r, (i0, i1) in enumerate(occupied_ranges(o, world)):
            S = ctx.sigma_share(X, i0, i1, r == 0)
            main += S[:, :n1]
            sats.append(S[:, n1:])
        got = np.concatenate([main] + sats, axis=1)
    ref = oadc.sigma_ref("EA", order, x, p.B, p.eps_occ, p.eps_vir, X)
    assert _rel(got, full).max() < 1e-12
    assert _rel(got, ref).max() < 1e-12


def test_share_rejects_other_kinds_and_ranges(gpu):
    p = make_problem(4, 6, 8, seed=66, sigma=0.1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=1.0) as ctx:
        X = random_vectors(ctx.N, 1, seed=1)
        with pytest.raises(gpu.AdcError) as e:
            ctx.sigma_share(X, 0, 2, True)
        assert e.value.code == -6
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=3, x=1.0) as ctx:
        X = random_vectors(ctx.N, 1, seed=1)
        with pytest.raises(gpu.AdcError) as e:
            ctx.sigma_share(X, 2, 5, True)
        assert e.value.code == -1
