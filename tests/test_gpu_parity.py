"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances:
* FP64 sigma: ||S - S_ref|| / ||S_ref|| <= 1e-12 per vector.
* BF16x3 sigma: <= 1e-4 per vector. Each FP64 operand is split into two BF16
  numbers (about 2^-17 relative representation error), three of the four
  partial products are kept (dropped term 2^-16 * 2^-16), and the tensor
  cores accumulate in FP32, whose rounding grows like sqrt(K) * 2^-24 for
  the longest inner sizes here (K <= 2e5 embedded terms): about 2e-5 in all,
  so 1e-4 leaves a factor of five.
* Sliced (FP64-accurate) tensor-core product and sigma: 1e-10. The digit
  products are exact in FP32; what remains is the truncation after about 40
  bits relative to the row and column maxima, about 1e-11 of the output norm
  for these value distributions, plus the FP64 combination.
* Eigenvalues: 1e-8 Eh (FP64 Davidson), 1e-6 Eh (mixed Davidson with FP64
  or sliced refinement).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle import adc as oadc  # noqa: E402
from oracle.fns import fns_density, fns_basis  # noqa: E402


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


# ---------------------------------------------------------------- GEMM kernels
@pytest.mark.parametrize("M,N,K", [(300, 70, 1000), (1, 1, 1), (65, 129, 17)])
def test_fp64_gemm(gpu, M, N, K):
    err, ms = gpu.diag_gemm(0, M, N, K, seed=3)
    assert err < 1e-14


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("m,nb,n", [(1, 1, 1), (8, 8, 4096), (13, 5, 20011), (40, 8, 70000), (64, 16, 33333),
                                     (97, 3, 5000), (33, 1, 1234567), (200, 12, 777)])
def test_davidson_block_kernels(gpu, which, m, nb, n):
    """The Davidson's FP64 block kernels (projections V^H T, 0; subspace
    combinations sum_i C[i][r] V[i], 1) equal the FP64 GEMM on ragged shapes:
    tiles of the short indices cut off, long vectors that are no multiple of
    the staged length, a single element."""
    err, ms = gpu.diag_blockops(which, m, nb, n, seed=11, reps=1)
    assert err < 1e-13, (which, m, nb, n, err)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (200, 40, 1000), (129, 130, 70), (1000, 300, 5000),
                                   (64, 8, 20000)])
def test_bf16x3_gemm(gpu, M, N, K):
    err, ms = gpu.diag_gemm(1, M, N, K, seed=5)
    assert err < 5e-5, err


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (200, 40, 1000), (129, 130, 70), (1000, 300, 5000),
                                   (64, 8, 20000)])
def test_bf16x6_gemm(gpu, M, N, K):
    """Six-product split: about 2^-24 per operand, but the tensor cores' FP32
    accumulation sets the floor (1e-6 to 1e-5 relative here, the same as for
    the three-product split), so the bound is the three-product one."""
    err, ms = gpu.diag_gemm(4, M, N, K, seed=5)
    assert err < 5e-5, err


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (200, 40, 1000), (129, 130, 70), (1000, 300, 5000),
                                   (130, 3, 70000), (300, 1, 129)])
def test_sliced_gemm(gpu, M, N, K):
    """Sliced FP64-accurate product (exact digit products in FP32, FP64
    combination); (130, 3, 70000) splits K for exactness."""
    err, ms = gpu.diag_gemm(5, M, N, K, seed=7)
    assert err < 1e-10, err


@pytest.mark.parametrize("cap", [0, 3 << 20, 1 << 20])
def test_sliced_setup_gemm_in_chunks(gpu, cap):
    """The setup's sliced route (48 bits) with operand chunks of `cap` bytes:
    A row blocks, B column blocks and, below one 128-row tile, inner splits
    whose FP64-accurate partial products add up in the output."""
    try:
        assert gpu.lib.adc_diag_set_sliced_cap(cap) == 0
        for M, N, K in ((300, 200, 3000), (129, 70, 9000)):
            err, ms = gpu.diag_gemm(6, M, N, K, seed=11)
            assert err < 1e-12, (M, N, K, err)
    finally:
        gpu.lib.adc_diag_set_sliced_cap(0)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (200, 40, 1000), (129, 130, 70), (1000, 300, 5000),
                                   (64, 8, 20000), (300, 1, 129)])
def test_grouped_gemm_one_job(gpu, M, N, K):
    """The grouped persistent launch with an autotuned tile width, one job."""
    err, ms = gpu.diag_gemm(2, M, N, K, seed=5)
    assert err < 5e-5, err


@pytest.mark.parametrize("M,N,K", [(1000, 300, 5000), (129, 130, 70), (4000, 64, 3000)])
def test_grouped_gemm_three_jobs(gpu, M, N, K):
    """Three jobs of different shapes in one launch, one of them split along K."""
    err, ms = gpu.diag_gemm(3, M, N, K, seed=9)
    assert err < 5e-5, err


# ---------------------------------------------------------------- sigma parity
CASES = [
    ("IP", 5, 37, 40, 3, 0.5, 11),
    ("IP", 2, 9, 7, 3, 1.0, 12),     # one occupied pair
    ("IP", 9, 20, 30, 2, 0.0, 13),
    ("IP", 8, 24, 96, 3, 1.0, 0),    # the small IP-ADC(3) workload
    ("EA", 6, 30, 64, 3, 0.5, 14),
    ("EA", 3, 2, 5, 3, 1.0, 15),     # one virtual pair
    ("EA", 4, 45, 50, 2, 0.0, 16),
    ("EA", 7, 33, 70, 3, 1.0, 17),
]


@pytest.mark.parametrize("kind,o,v,Q,order,x,seed", CASES)
def test_sigma_parity(gpu, kind, o, v, Q, order, x, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.08)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x) as ctx:
        n1, n2 = oadc.dims(kind, o, v)
        assert (ctx.n1, ctx.n2) == (n1, n2)
        X = random_vectors(ctx.N, 3, seed=seed + 100)
        amp = oadc.Amplitudes(p.B, p.eps_occ, p.eps_vir, second_order=(order == 3))
        ref = oadc.sigma_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, X, amp=amp)
        # host pointers
        S = ctx.sigma(X, "fp64")
        assert _rel(S, ref).max() < 1e-12
        # device pointers, single vector
        Xd = torch.from_numpy(X[1:2].copy()).cuda()
        Sd = ctx.sigma(Xd, "fp64").cpu().numpy()
        assert _rel(Sd, ref[1:2]).max() < 1e-12
        Sm = ctx.sigma(X, "bf16x3")
        assert _rel(Sm, ref).max() < 1e-4
        Sm6 = ctx.sigma(X, "bf16x6")
        assert _rel(Sm6, ref).max() < 1e-4, _rel(Sm6, ref).max()
        Ss = ctx.sigma(X, "sliced")
        assert _rel(Ss, ref).max() < 1e-10, _rel(Ss, ref).max()
        # the intermediate refinement step: digits for about 24 bits
        Ss24 = ctx.sigma(X, "sliced24")
        assert _rel(Ss24, ref).max() < 2e-6, _rel(Ss24, ref).max()
        d = ctx.diagonal()
        dref = oadc.diagonal_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, amp=amp)
        assert np.abs(d - dref).max() < 1e-12 * max(1.0, np.abs(dref).max())
        mb = oadc.main_block(kind, amp) if order == 3 else None
        M11 = ctx.main_block()
        if mb is not None:
            ref11 = mb[0] + mb[2] + x * mb[3]
            assert np.abs(M11 - ref11).max() < 1e-12 * np.abs(ref11).max()


@pytest.mark.parametrize("kind,o,v,Q,order,x,seed,k", [
    ("EA", 6, 30, 64, 3, 0.5, 14, 3), ("EA", 4, 45, 50, 2, 0.0, 16, 2), ("EA", 7, 33, 70, 3, 1.0, 17, 9),
    ("IP", 8, 24, 96, 3, 1.0, 0, 4), ("IP", 9, 20, 30, 2, 0.0, 13, 1), ("IP", 5, 37, 40, 3, 0.5, 11, 7)])
def test_grouped_split_sigma(gpu, kind, o, v, Q, order, x, seed, k):
    """The BF16x3 product with all tensor-core terms in one grouped launch (default)
    against one launch per term and against the oracle: both are the same three-product
    split, so they differ only by the FP32 summation order of the tiles."""
    p = make_problem(o, v, Q, seed=seed, sigma=0.08)
    X = random_vectors(oadc.dims(kind, o, v)[0] + oadc.dims(kind, o, v)[1], k, seed=seed + 200)
    ref = oadc.sigma_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, X)
    out = {}
    for grouped in (True, False):
        with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x, grouped_sigma=grouped) as ctx:
            out[grouped] = ctx.sigma(X, "bf16x3")
            # repeated calls reuse the job table and the packed operands
            assert np.array_equal(ctx.sigma(X, "bf16x3"), out[grouped])
    assert _rel(out[True], ref).max() < 1e-4
    assert _rel(out[True], out[False]).max() < 1e-5


@pytest.mark.parametrize("o,v,Q,x,chunk", [(5, 12, 30, 1.0, 2), (4, 9, 20, 0.5, 4)])
def test_ip_coupling_intermediate_in_chunks(gpu, o, v, Q, x, chunk):
    """IP third order: the (ea|fk) block of the second-order coupling formed in
    chunks of a (here `chunk` virtual indices per chunk, a ragged last one),
    equal to the oracle and to the context built in one chunk."""
    p = make_problem(o, v, Q, seed=71, sigma=0.08)
    X = random_vectors(o + oadc.dims("IP", o, v)[1], 3, seed=72)
    ref = oadc.sigma_ref("IP", 3, x, p.B, p.eps_occ, p.eps_vir, X)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=x) as c1:
        S1 = c1.sigma(X, "fp64")
    try:
        assert gpu.lib.adc_diag_set_setup_chunk(chunk * o * v * v) == 0
        with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=x) as c2:
            S2 = c2.sigma(X, "fp64")
    finally:
        gpu.lib.adc_diag_set_setup_chunk(0)
    assert _rel(S2, ref).max() < 1e-12
    assert _rel(S2, S1).max() < 1e-13


def test_sigma_zero_vectors_and_k0(gpu):
    p = make_problem(4, 10, 12, seed=2, sigma=0.1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=3, x=1.0) as ctx:
        X = np.zeros((2, ctx.N), np.complex128)
        assert np.abs(ctx.sigma(X, "fp64")).max() == 0.0
        assert np.abs(ctx.sigma(X, "bf16x3")).max() == 0.0
        assert np.abs(ctx.sigma(X, "sliced")).max() == 0.0
        assert gpu.lib.adc_sigma(ctx._h, None, None, 0, 0) == 0
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=0.5) as ctx:
        X = np.zeros((1, ctx.N), np.complex128)
        assert np.abs(ctx.sigma(X, "sliced")).max() == 0.0


# ---------------------------------------------------------------- eigenvalues
def test_ip_adc3_small_workload_davidson(gpu):
    p = make_problem(8, 24, 96, seed=0, sigma=0.05, occ_range=(-2.0, -0.5), vir_range=(0.2, 3.0))
    M = oadc.explicit_matrix("IP", 3, 1.0, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:4]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=1.0) as ctx:
        om, Y, e64, st, rc = ctx.davidson(4, tol=1e-8, precision="fp64")
        assert rc == 0
        assert np.abs(om - w).max() < 1e-8
        assert np.all(e64 <= 1e-8)
        assert np.abs(Y.conj() @ Y.T - np.eye(4)).max() < 1e-10
        R = Y @ M.T - om[:, None] * Y
        assert np.linalg.norm(R, axis=1).max() < 1e-7
        om2, _, e2, st2, rc2 = ctx.davidson(4, tol=1e-8, precision="bf16x3", want_vectors=False)
        assert rc2 == 0 and np.abs(om2 - w).max() < 1e-8
        assert st2["sigma_calls_fp64"] > 0


def test_mixed_davidson_preconditioned_corrections_in_subspace(gpu):
    """IP-ADC(2) case whose preconditioned corrections fall into the subspace
    in the split-precision phase; the solver must still reach the FP64 tolerance."""
    p = make_problem(5, 14, 28, seed=54, sigma=0.06, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    M = oadc.explicit_matrix("IP", 2, 0.0, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:3]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=2, x=0.0) as ctx:
        om, _, e64, st, rc = ctx.davidson(3, tol=1e-7, precision="bf16x3", want_vectors=False)
        assert rc == 0 and np.all(e64 <= 1e-7)
        assert np.abs(om - w).max() < 1e-8


@pytest.mark.parametrize("kind,o,v,Q,x,prec", [("EA", 6, 30, 64, 0.5, "bf16x3"), ("IP", 7, 26, 50, 0.5, "bf16x3"),
                                              ("EA", 6, 30, 64, 0.5, "bf16x6")])
def test_mixed_davidson_refined(gpu, kind, o, v, Q, x, prec):
    p = make_problem(o, v, Q, seed=21, sigma=0.06, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    M = oadc.explicit_matrix(kind, 3, x, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:4]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=x) as ctx:
        om, Y, e64, st, rc = ctx.davidson(4, tol=1e-7, precision=prec)
        assert rc == 0
        assert np.abs(om - w).max() < 1e-6
        assert np.all(e64 <= 1e-7)
        R = Y @ M.T - om[:, None] * Y
        assert np.linalg.norm(R, axis=1).max() < 1e-6


@pytest.mark.parametrize("kind,o,v,Q,x", [("EA", 6, 30, 64, 0.5), ("IP", 7, 26, 50, 0.5), ("EA", 5, 24, 40, 1.0)])
def test_mixed_davidson_sliced_refinement(gpu, kind, o, v, Q, x):
    """Mixed Davidson whose refinement products (FP64 base of the Ritz vectors,
    final residual check) are the sliced tensor-core product."""
    p = make_problem(o, v, Q, seed=22, sigma=0.06, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    M = oadc.explicit_matrix(kind, 3, x, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:4]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=x, refine="sliced") as ctx:
        om, Y, e64, st, rc = ctx.davidson(4, tol=1e-7, precision="bf16x3")
        assert rc == 0
        assert st["sigma_calls_fp64"] > 0
        assert np.abs(om - w).max() < 1e-6
        assert np.all(e64 <= 1e-7)
        R = Y @ M.T - om[:, None] * Y
        assert np.linalg.norm(R, axis=1).max() < 1e-6


@pytest.mark.parametrize("kind,o,v,Q,order,x,seed", [("EA", 8, 40, 80, 3, 0.5, 41), ("IP", 12, 30, 80, 3, 1.0, 42),
                                                     ("EE", 6, 20, 40, 3, 0.4, 43), ("EA", 6, 36, 60, 2, 0.0, 44),
                                                     ("IP", 6, 20, 600, 3, 1.0, 45), ("EA", 5, 21, 560, 3, 0.5, 46),
                                                     ("EE", 4, 10, 520, 3, 0.4, 47), ("EE", 6, 16, 520, 2, 0.0, 48)])
def test_sliced_setup(gpu, kind, o, v, Q, order, x, seed):
    """adc_init with opts.setup = ADC_PREC_SLICED: the setup's contractions of at
    least 2^24 flops and inner size 512 run as the sliced product (about 48
    bits); sigma, diagonal and main block match the oracle to 1e-11 relative
    (FP64 setup: 1e-12). The routes adc_init took are counted: with naux >= 512
    every kind's integral assembly over the Cholesky index goes through the
    sliced product, a third or more of the setup's flops at these sizes (the
    EE setup's many products below 2^24 flops stay on the FP64 cores)."""
    p = make_problem(o, v, Q, seed=seed, sigma=0.08)
    kw = dict(kind=kind, order=order, x=x)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, setup="sliced", **kw) as ctx:
        X = random_vectors(ctx.N, 2, seed=seed + 1)
        S = ctx.sigma(X, "fp64")
        d = ctx.diagonal()
        M11 = ctx.main_block()
        routes = ctx.setup_routes()
    if kind == "EE":
        from oracle import adc_ee
        M = adc_ee.explicit_matrix(order, x, p.B, p.eps_occ, p.eps_vir)
        ref = X @ M.T
        dref = np.real(np.diag(M))
        m11 = M[:ctx.n1, :ctx.n1]
    else:
        amp = oadc.Amplitudes(p.B, p.eps_occ, p.eps_vir, second_order=(order == 3))
        ref = oadc.sigma_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, X, amp=amp)
        dref = oadc.diagonal_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, amp=amp)
        m11 = oadc.explicit_matrix(kind, order, x, p.B, p.eps_occ, p.eps_vir)[:ctx.n1, :ctx.n1]
    assert _rel(S, ref).max() < 1e-11, _rel(S, ref).max()
    assert np.abs(d - dref).max() < 1e-11 * max(1.0, np.abs(dref).max())
    assert np.abs(M11 - m11).max() < 1e-11 * max(1.0, np.abs(m11).max())
    if Q >= 512:
        total = routes["flops_sliced"] + routes["flops_fp64"]
        assert routes["n_sliced"] >= 1 and routes["flops_sliced"] >= total / 3, routes


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-4), ("sliced", 1e-10)])
def test_tensor_core_wait_gives_up_and_context_recovers(gpu, prec, tol):
    """A pipeline wait of the tensor-core kernels that runs out: the wait limit
    is lowered to 1 ns through the test hook, so a wait gives up long before
    the copies and MMAs it waits for finish. The kernels drain what they have
    in flight and return; the call reports ADC_ERR_TIMEOUT (-5). With the
    limit restored the next call on the same context gives the normal result
    (against the oracle). The operand copies and tile widths are built at the
    normal limit first."""
    p = make_problem(6, 60, 50, seed=51, sigma=0.08)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=3, x=0.5) as ctx:
        X = random_vectors(ctx.N, 2, seed=52)
        first = ctx.sigma(X, prec)
        assert gpu.lib.adc_diag_set_wait_ns(1) == 0
        try:
            with pytest.raises(gpu.AdcError) as ei:
                ctx.sigma(X, prec)
            assert ei.value.code == -5, ei.value
        finally:
            assert gpu.lib.adc_diag_set_wait_ns(0) == 0
        again = ctx.sigma(X, prec)
    ref = oadc.sigma_ref("EA", 3, 0.5, p.B, p.eps_occ, p.eps_vir, X)
    assert _rel(again, first).max() < 1e-14
    assert _rel(again, ref).max() < tol


@pytest.mark.parametrize("kind,prec", [("EA", "fp64"), ("IP", "fp64"), ("EA", "bf16x3")])
def test_davidson_olsen_correction(gpu, kind, prec):
    """Olsen's correction vectors (opts.correction = 1) reach the dense oracle's
    lowest roots like the plain preconditioned residuals."""
    p = make_problem(5, 14, 24, seed=57, sigma=0.08, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    M = oadc.explicit_matrix(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:4]
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=0.5, correction="olsen",
                     refine="sliced") as ctx:
        om, Y, e64, st, rc = ctx.davidson(4, tol=1e-8, precision=prec)
    assert rc == 0
    assert np.abs(om - w).max() < 1e-8
    R = Y @ M.T - om[:, None] * Y
    assert np.linalg.norm(R, axis=1).max() < 1e-7


def test_davidson_noconv_returns_best(gpu):
    p = make_problem(5, 12, 20, seed=3, sigma=0.08)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=1.0) as ctx:
        om, _, e64, st, rc = ctx.davidson(3, tol=1e-12, max_iter=1, precision="fp64", raise_on_noconv=False)
        assert rc == -4
        assert np.all(np.isfinite(om)) and np.all(e64 > 0)


# ---------------------------------------------------------------- natural spinors (Eqs. 25-30)
def test_fns_density_and_truncation(gpu):
    o, v, Q = 6, 30, 64
    p = make_problem(o, v, Q, seed=31, sigma=0.06)
    Dref = fns_density(p.B, p.eps_occ, p.eps_vir)
    eta_r, V_r, nk_r, U_r, e_r = fns_basis(Dref, p.eps_vir, -1.0)
    crit = float(np.sqrt(eta_r[9] * eta_r[10]))  # inside the gap between the 10th and 11th
    eta_r, V_r, nk_r, U_r, e_r = fns_basis(Dref, p.eps_vir, crit)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=2) as ctx:
        r = ctx.fns_density(crit)
    assert np.abs(r["D"] - Dref).max() < 1e-12 * np.abs(Dref).max()
    assert np.abs(r["eta"] - eta_r).max() < 1e-12 * eta_r.max()
    assert r["n_keep"] == nk_r == 10
    assert np.abs(r["eps_new"] - e_r).max() < 1e-10
    P_gpu = r["U"] @ r["U"].conj().T
    P_ref = U_r @ U_r.conj().T
    assert np.abs(P_gpu - P_ref).max() < 1e-9
    V = r["V"]
    assert np.abs(V.conj().T @ V - np.eye(v)).max() < 1e-10


# ---------------------------------------------------------------- errors
def test_error_codes(gpu):
    p = make_problem(4, 10, 8, seed=4, sigma=0.1)
    Bbad = p.B.copy()
    Bbad[0, 1, 2] += 0.01
    with pytest.raises(gpu.AdcError) as e:
        gpu.Context(Bbad, p.eps_occ, p.eps_vir, kind="IP")
    assert e.value.code == -1
    with pytest.raises(gpu.AdcError) as e:
        gpu.Context(p.B, p.eps_occ + 10.0, p.eps_vir, kind="IP")
    assert e.value.code == -1
    with pytest.raises(gpu.AdcError) as e:
        gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", mem_limit=1024)
    assert e.value.code == -2
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP") as ctx:
        with pytest.raises(gpu.AdcError) as e:
            ctx.sigma(np.zeros((1, ctx.N), np.complex128), precision=7)
        assert e.value.code == -1


def test_fns_transform_and_invariance(gpu):
    from oracle.fns import transform_cholesky
    o, v, Q = 5, 22, 40
    p = make_problem(o, v, Q, seed=33, sigma=0.07)
    Dref = fns_density(p.B, p.eps_occ, p.eps_vir)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=3, x=1.0) as ctx:
        full = ctx.fns_density(-1.0)      # keep every natural spinor
        assert full["n_keep"] == v
        Bf = ctx.fns_transform(full["U"])
        trunc = ctx.fns_density(float(np.sort(full["eta"])[::-1][11]))
        Bt = ctx.fns_transform(trunc["U"])
        w_can, _, _, _, _ = ctx.davidson(3, tol=1e-9, precision="fp64", want_vectors=False)
    # transformation matches the oracle for the same U
    assert np.abs(Bf - transform_cholesky(p.B, o, full["U"])).max() < 1e-13
    assert np.abs(Bt - transform_cholesky(p.B, o, trunc["U"])).max() < 1e-13
    assert Bt.shape == (Q, o + 12, o + 12)
    # keeping every natural spinor is a unitary rotation of the virtuals with the
    # Fock matrix semicanonical (diagonal), so the IP spectrum is unchanged
    with gpu.Context(Bf, p.eps_occ, full["eps_new"], kind="IP", order=3, x=1.0) as c2:
        w_fns, _, _, _, _ = c2.davidson(3, tol=1e-9, precision="fp64", want_vectors=False)
    assert np.abs(w_fns - w_can).max() < 1e-8
