"""Multi-rank dataflow of one EA problem split by the satellites' occupied index,
on CPU processes over gloo (world sizes 2 and 3).

Each rank holds the 1p rows and the 2p1h rows of its occupied range. Its
local products stand in for its GPU's share (adc_sigma_share) and are built
from the oracle's explicit blocks (Sec. 2.1): the coupling of its
satellites, their zeroth-order diagonal and ring rows against the gathered
trial block, and the ladder, diagonal in the occupied index, against its own
rows only. paper_2511_21640_gb300.shard supplies the split, the all-gather of
the trial block, the all-reduce of the partial 1p rows and of the subspace
projections. The sharded sigma and projections must equal the unsharded
oracle sigma and V^H S."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from synthetic import make_problem, random_vectors  # noqa: E402
from oracle import adc  # noqa: E402
from oracle.integrals import eri  # noqa: E402

O, V, Q, X_SCALE = 5, 6, 8, 0.5


@pytest.fixture(scope="module", autouse=True)
def _library():
    # the shard module lives in the package, whose import loads the library
    from conftest import build_library
    build_library()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _blocks():
    p = make_problem(O, V, Q, seed=61, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    bl = adc.Blocks("EA", p.B, p.eps_occ, p.eps_vir)
    M11 = bl.M11[0] + bl.M11[2] + X_SCALE * bl.M11[3]
    C = bl.M12[1] + X_SCALE * bl.M12[2]
    iu, ju = np.triu_indices(V, 1)
    vvvv = eri(p.B, O, "vvvv")[iu, ju][:, iu, ju]              # <ab||cd>, a<b, c<d
    L = np.kron(np.eye(O), vvvv)                                # ladder: diagonal in the occupied index
    ring = bl.M22[1] - L                                        # the rest of the first-order block
    return p, M11, C, np.diag(bl.M22[0]), L, ring


def _rank_main(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2511_21640_gb300.shard import OccupiedSplit, sharded_projection, sharded_sigma
        p, M11, C, d0, L, ring = _blocks()
        sp = OccupiedSplit(O, V, world, rank)
        n1 = sp.n1

        def share(Xw, i0, i1, with_main):
            X = Xw.numpy()
            X1, X2 = X[:, :n1], X[:, n1:]
            blk = slice(i0 * sp.pv, i1 * sp.pv)
            main = X2[:, blk] @ C[:, blk].T + (X1 @ M11.T if with_main else 0.0)
            sat = (X1 @ C[:, blk].conj() + d0[blk] * X2[:, blk] + X_SCALE * X2 @ ring[blk, :].T
                   + X_SCALE * X2[:, blk] @ L[blk, blk].T)
            return torch.from_numpy(np.concatenate([main, sat], axis=1))

        def gram(A, B):
            return A.conj() @ B.T

        X = torch.from_numpy(random_vectors(sp.N, 3, seed=62))
        Vs = torch.from_numpy(random_vectors(sp.N, 4, seed=63))
        S_local = sharded_sigma(sp, sp.local_of(X), share)
        ref = adc.sigma_ref("EA", 3, X_SCALE, p.B, p.eps_occ, p.eps_vir, X.numpy())
        ref_local = sp.local_of(torch.from_numpy(ref)).numpy()
        assert np.abs(S_local.numpy() - ref_local).max() < 1e-12 * np.abs(ref).max(), rank
        G = sharded_projection(sp, sp.local_of(Vs), S_local, gram)
        G_ref = Vs.numpy().conj() @ ref.T
        assert np.abs(G.numpy() - G_ref).max() < 1e-12 * np.abs(G_ref).max(), rank
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sigma_and_projections_equal_unsharded(world):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port()), nprocs=world, join=True)


def test_occupied_ranges_cover_once():
    from paper_2511_21640_gb300.shard import OccupiedSplit, occupied_ranges
    for nocc in (1, 5, 40):
        for world in (1, 2, 3, 8):
            r = occupied_ranges(nocc, world)
            assert r[0][0] == 0 and r[-1][1] == nocc
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1
            n_local = sum(OccupiedSplit(nocc, 7, world, k).n_local - 7 for k in range(world))
            assert n_local == nocc * 21
