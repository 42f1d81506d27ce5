"""adc_sigma_noalloc: the FP64 sigma product for callers that cannot allocate
GPU memory during the call (their device memory belongs to another
allocator, or cudaMalloc would stall or fail them mid-run). The entry point
keeps its intermediates in a fixed __device__ array instead; its results must
equal adc_sigma's FP64 results on consecutive calls (the array is reused, so
a second call must not see stale data from the first). On tiny IP and EA
problems they must also equal the CPU oracle's explicit matrix times X, so a
fault shared by both GPU entry points cannot hide behind their agreement."""
import ctypes

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


def _noalloc(m, ctx, Xd, Sd):
    ctx.sync()
    torch.cuda.synchronize()
    rc = m.lib.adc_sigma_noalloc(ctx._h, ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Sd.data_ptr()),
                                 Xd.shape[0])
    ctx.sync()
    return rc


@pytest.mark.parametrize("kind,o,v,Q,order,x", [("EA", 5, 21, 30, 3, 0.5), ("IP", 6, 17, 25, 3, 1.0),
                                                ("EA", 4, 12, 10, 2, 0.0)])
def test_noalloc_matches_sigma_on_two_calls(gpu, kind, o, v, Q, order, x):
    p = make_problem(o, v, Q, seed=41, sigma=0.08)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x) as ctx:
        for call, seed in enumerate((1, 2)):
            X = torch.from_numpy(random_vectors(ctx.N, 3, seed=seed)).cuda()
            ref = ctx.sigma(X, "fp64").cpu().numpy()
            S = torch.full_like(X, complex(np.nan, np.nan))
            assert _noalloc(gpu, ctx, X, S) == 0, gpu.lib.adc_last_error(ctx._h)
            got = S.cpu().numpy()
            err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert err.max() < 1e-12, (call, err)


def test_noalloc_rejects_host_pointers_and_oversize(gpu):
    p = make_problem(4, 30, 12, seed=42, sigma=0.08)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=3, x=1.0) as ctx:
        Xh = random_vectors(ctx.N, 1, seed=3)
        Sh = np.empty_like(Xh)
        rc = gpu.lib.adc_sigma_noalloc(ctx._h, ctypes.c_void_p(Xh.ctypes.data), ctypes.c_void_p(Sh.ctypes.data), 1)
        assert rc == -1
        # 2 k o v^2 complex elements above the 2^22-element array
        k = (1 << 22) // (2 * 4 * 30 * 30) + 1
        X = torch.zeros((k, ctx.N), dtype=torch.complex128, device="cuda")
        S = torch.zeros_like(X)
        assert _noalloc(gpu, ctx, X, S) == -1
        assert b"scratch" in gpu.lib.adc_last_error(ctx._h)


@pytest.mark.parametrize("kind,o,v,Q,x", [("IP", 4, 7, 9, 1.0), ("EA", 3, 8, 10, 0.5)])
def test_noalloc_matches_oracle_explicit_matrix(gpu, kind, o, v, Q, x):
    p = make_problem(o, v, Q, seed=43, sigma=0.1)
    M = oadc.explicit_matrix(kind, 3, x, p.B, p.eps_occ, p.eps_vir)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=x) as ctx:
        assert ctx.N == M.shape[0]
        for call, seed in enumerate((5, 6)):
            Xh = random_vectors(ctx.N, 2, seed=seed)
            ref = Xh @ M.T
            X = torch.from_numpy(Xh).cuda()
            S = torch.full_like(X, complex(np.nan, np.nan))
            assert _noalloc(gpu, ctx, X, S) == 0, gpu.lib.adc_last_error(ctx._h)
            got = S.cpu().numpy()
            err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert err.max() < 1e-12, (call, err)
