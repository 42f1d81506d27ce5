"""Batches of independent IP/EA problems: grouped persistent tensor-core
launch, graph capture and replay, lockstep Davidson, wave scheduler.

Tolerances as in test_gpu_parity: 1e-4 per vector for split-precision sigma
against the oracle, 1e-12 for FP64; eigenvalues 1e-6 Eh after FP64
refinement (1e-8 Eh against the dense oracle where the matrix is explicit).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle import adc as oadc  # noqa: E402

# uneven problems: kinds, orders, x, one-pair edge cases, ragged sizes
SET = [
    ("EA", 6, 30, 64, 3, 0.5, 31),
    ("IP", 5, 37, 40, 3, 1.0, 32),
    ("EA", 3, 2, 5, 3, 1.0, 33),
    ("IP", 9, 20, 30, 2, 0.0, 34),
    ("EA", 7, 41, 70, 3, 0.3, 35),
    ("IP", 2, 9, 7, 3, 0.5, 36),
]


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


def _contexts(gpu, cases):
    out = []
    for kind, o, v, Q, order, x, seed in cases:
        p = make_problem(o, v, Q, seed=seed, sigma=0.08)
        out.append((p, gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x)))
    return out


def test_batched_sigma_matches_oracle_and_replays(gpu):
    pcs = _contexts(gpu, SET)
    ks = [3, 1, 2, 4, 3, 2]
    Xh = [random_vectors(c.N, k, seed=200 + i) for i, ((p, c), k) in enumerate(zip(pcs, ks))]
    refs = []
    for (p, c), X, case in zip(pcs, Xh, SET):
        kind, o, v, Q, order, x, seed = case
        amp = oadc.Amplitudes(p.B, p.eps_occ, p.eps_vir, second_order=(order == 3))
        refs.append(oadc.sigma_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, X, amp=amp))
    Xd = [torch.from_numpy(X).cuda() for X in Xh]
    with gpu.Batch([c for _, c in pcs]) as b:
        Sd = [torch.empty_like(X) for X in Xd]
        outs = []
        for _ in range(3):  # direct, captured, replayed (same pointers each time)
            outs.append([S.clone() for S in b.sigma(Xd, "bf16x3", outs=Sd)])
        info = b.info()
        assert info["batches"] == 3 and info["graphs_captured"] == 1 and info["graph_launches"] == 2
        assert info["direct_launches"] == 1 and info["tuned_shapes"] >= 1
        for S, R in zip(outs[0], refs):
            assert _rel(S.cpu().numpy(), R).max() < 1e-4
        for r in (1, 2):  # the graph replays the same kernels on the same data
            for S0, S1 in zip(outs[0], outs[r]):
                assert torch.equal(S0, S1)
        # against the per-problem split-precision product (other tiles, same splits)
        for (p, c), X, S in zip(pcs, Xh, outs[0]):
            Sc = c.sigma(X, "bf16x3")
            assert _rel(S.cpu().numpy(), Sc).max() < 5e-5
        # FP64 through the batch equals the per-problem FP64 product bit for bit
        S64 = b.sigma(Xd, "fp64", outs=Sd)
        for (p, c), X, S, R in zip(pcs, Xh, S64, refs):
            assert np.array_equal(S.cpu().numpy(), c.sigma(X, "fp64"))
            assert _rel(S.cpu().numpy(), R).max() < 1e-12
        # a batch where one problem sits out (k = 0) and graphs switched off
        b.use_graphs(False)
        Xz = list(Xd)
        Xz[2] = Xd[2][:0]
        Sz = b.sigma(Xz, "bf16x3")
        for i in (0, 1, 3, 4, 5):
            assert _rel(Sz[i].cpu().numpy(), refs[i]).max() < 1e-4
    for _, c in pcs:
        c.close()


def test_batched_davidson_matches_dense(gpu):
    cases = [("EA", 6, 30, 64, 3, 0.5, 41), ("IP", 7, 26, 50, 3, 0.5, 42), ("EA", 5, 22, 40, 2, 0.0, 43),
             ("IP", 6, 18, 30, 3, 1.0, 44)]
    pcs = []
    dense = []
    for kind, o, v, Q, order, x, seed in cases:
        p = make_problem(o, v, Q, seed=seed, sigma=0.06, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
        M = oadc.explicit_matrix(kind, order, x, p.B, p.eps_occ, p.eps_vir)
        dense.append(np.linalg.eigvalsh(M)[:4])
        pcs.append(gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x))
    with gpu.Batch(pcs) as b:
        om, e64, status, st, rc = b.davidson(4, tol=1e-7, precision="bf16x3")
        assert rc == 0 and np.all(status == 0), (status, e64, st)
        for i, w in enumerate(dense):
            assert np.abs(om[i] - w).max() < 1e-8
            assert np.all(e64[i] <= 1e-7)
        info = b.info()
        assert info["batches"] > 0 and info["graph_launches"] > 0
        om64, e6, s6, _, rc6 = b.davidson(4, tol=1e-7, precision="fp64")
        assert rc6 == 0 and np.abs(om64 - om).max() < 1e-8
    for c in pcs:
        c.close()


def test_batch_solve_waves(gpu):
    """Raw problems through the scheduler, forced into several waves."""
    cases = [("EA", 5, 24, 40, 3, 0.5, 51), ("IP", 6, 20, 36, 3, 0.5, 52), ("EA", 4, 16, 30, 3, 0.5, 53),
             ("IP", 5, 14, 28, 2, 0.0, 54), ("EA", 3, 12, 20, 3, 1.0, 55)]
    probs = []
    dense = []
    for kind, o, v, Q, order, x, seed in cases:
        p = make_problem(o, v, Q, seed=seed, sigma=0.06, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0),
                         kind=kind, order=order, x=x)
        probs.append(p)
        M = oadc.explicit_matrix(kind, order, x, p.B, p.eps_occ, p.eps_vir)
        dense.append(np.linalg.eigvalsh(M)[:3])
    plan = gpu.batch_plan([dict(kind=p.kind, nocc=p.nocc, nvir=p.nvir, naux=p.naux, order=p.order, x=p.x)
                           for p in probs], 3, 1)
    budget = int(plan[3].max() * 1.5)  # at most two of the largest together
    nw = gpu.batch_plan([dict(kind=p.kind, nocc=p.nocc, nvir=p.nvir, naux=p.naux, order=p.order, x=p.x)
                         for p in probs], 3, budget)[0]
    assert nw >= 2
    om, e64, status, info, rc = gpu.batch_solve(probs, 3, tol=1e-7, mem_budget=budget, init_lanes=2)
    assert rc == 0 and np.all(status == 0)
    assert info["waves"] == nw
    for i, w in enumerate(dense):
        assert np.abs(om[i] - w).max() < 1e-8


def test_batch_rejects_ee_mixed(gpu):
    p = make_problem(3, 6, 10, seed=5, sigma=0.08)
    q = make_problem(4, 10, 12, seed=6, sigma=0.08)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=2) as ce, \
            gpu.Context(q.B, q.eps_occ, q.eps_vir, kind="EA", order=3, x=0.5) as ca:
        with gpu.Batch([ce, ca]) as b:
            Xs = [torch.from_numpy(random_vectors(c.N, 1, seed=9)).cuda() for c in (ce, ca)]
            with pytest.raises(gpu.AdcError) as ei:
                b.sigma(Xs, "bf16x3")
            assert ei.value.code == -6
            S = b.sigma(Xs, "fp64")
            assert np.array_equal(S[0].cpu().numpy(), ce.sigma(Xs[0].cpu().numpy(), "fp64"))
