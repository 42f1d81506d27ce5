"""The integral-direct EA ladder (opts.ladder): the four-external integrals
<ab||cd> of the 2p1h block formed from the Cholesky vectors in chunks inside
every product (Sec. 2.5, Eq. 43 and the paragraph after it) instead of stored.
Its sigma must equal the stored path's and the oracle's in every precision,
on sizes of one and several chunks, and its Davidson roots the dense oracle's.
Tolerances as in test_gpu_parity (FP64 1e-12, sliced 1e-10, BF16x3 1e-4 per
vector)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle import adc as oadc  # noqa: E402
from oracle import rows as orows  # noqa: E402


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


def _pair(p, q, n):
    return p * n - p * (p + 1) // 2 + (q - p - 1)


@pytest.mark.parametrize("order,x", [(3, 0.5), (3, 1.0)])
def test_direct_ladder_small_against_oracle(gpu, order, x):
    o, v, Q = 4, 12, 20
    p = make_problem(o, v, Q, seed=101, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    ref_S = None
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=order, x=x, ladder="direct",
                     refine="sliced") as ctx:
        assert ctx.direct_ladder()
        X = random_vectors(ctx.N, 3, seed=102)
        ref_S = oadc.sigma_ref("EA", order, x, p.B, p.eps_occ, p.eps_vir, X)
        assert _rel(ctx.sigma(X, "fp64"), ref_S).max() < 1e-12
        assert _rel(ctx.sigma(X, "sliced"), ref_S).max() < 1e-10
        assert _rel(ctx.sigma(X, "bf16x3"), ref_S).max() < 1e-4
        M = oadc.explicit_matrix("EA", order, x, p.B, p.eps_occ, p.eps_vir)
        w = np.linalg.eigvalsh(M)[:3]
        om, _, _, _, rc = ctx.davidson(3, tol=1e-8, precision="fp64", want_vectors=False)
        assert rc == 0 and np.abs(om - w).max() < 1e-8
        om, _, _, _, rc = ctx.davidson(3, tol=1e-7, precision="bf16x3", want_vectors=False)
        assert rc == 0 and np.abs(om - w).max() < 1e-6
        # the allocation-free product needs the stored block
        Xd = torch.from_numpy(X).cuda()
        Sd = torch.empty_like(Xd)
        ctx.sync()
        rc = gpu.lib.adc_sigma_noalloc(ctx._h, ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Sd.data_ptr()), 3)
        assert rc == -6


def test_direct_ladder_several_chunks_equals_stored(gpu):
    """v = 110: the assembly runs in three chunks of the first virtual index."""
    o, v, Q, x = 3, 110, 24, 0.7
    p = make_problem(o, v, Q, seed=103, sigma=0.08, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    kw = dict(kind="EA", order=3, x=x)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, ladder="stored", **kw) as cs:
        assert not cs.direct_ladder()
        X = random_vectors(cs.N, 3, seed=104)
        S64 = cs.sigma(X, "fp64")
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, ladder="direct", **kw) as cd:
        assert cd.direct_ladder()
        D64 = cd.sigma(X, "fp64")
        Dsl = cd.sigma(X, "sliced")
        Dmx = cd.sigma(X, "bf16x3")
    assert _rel(D64, S64).max() < 1e-12
    assert _rel(Dsl, S64).max() < 1e-10
    assert _rel(Dmx, S64).max() < 1e-4
    pv = v * (v - 1) // 2
    sel = [(0, 0, 1), (2, 108, 109), (1, 37, 90), (0, 54, 55)]
    R = orows.ea_satellite_rows(p.B, p.eps_occ, p.eps_vir, 3, x, X, sel)
    idx = [v + k * pv + _pair(d, e, v) for k, d, e in sel]
    rms = float(np.sqrt(np.mean(np.abs(S64) ** 2)))
    assert np.abs(D64[:, idx] - R).max() < 1e-10 * rms


def test_direct_setup_ip_against_oracle(gpu):
    """IP: the four-virtual integrals enter only the second-order amplitudes'
    ladder intermediate, formed in chunks by the integral-direct setup."""
    o, v, Q = 5, 11, 20
    p = make_problem(o, v, Q, seed=105, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=1.0, ladder="direct") as ctx:
        assert ctx.direct_ladder()
        X = random_vectors(ctx.N, 2, seed=106)
        ref = oadc.sigma_ref("IP", 3, 1.0, p.B, p.eps_occ, p.eps_vir, X)
        assert _rel(ctx.sigma(X, "fp64"), ref).max() < 1e-12
        assert _rel(ctx.sigma(X, "sliced"), ref).max() < 1e-10
        assert _rel(ctx.sigma(X, "bf16x3"), ref).max() < 1e-4
