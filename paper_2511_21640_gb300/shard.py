"""One EA problem split across ranks by the occupied index of its satellites.

The 2p1h amplitudes X_j,(a<b) of an EA-ADC problem (Sec. 2.1, Eqs. 3-4) are
distributed over the ranks of a process group in contiguous ranges of their
occupied index j; every rank keeps a copy of the 1p amplitudes X_a. A sigma
product (Eq. 10) then takes three steps:

1. an all-gather of the ranks' satellite rows: the ring term and the coupling
   reach every j, so each rank needs the whole trial block;
2. each rank's share on its own GPU (``Context.sigma_share``, the C entry
   point ``adc_sigma_share``): the complete satellite rows of its j range (the
   ladder is diagonal in j) and the partial 1p rows of its satellites'
   coupling, one rank adding M11 X1;
3. an all-reduce (sum) of the partial 1p rows.

The Davidson projections V^H S of distributed vectors are partial sums over
each rank's rows (the 1p rows counted once), all-reduced.

Host logic only: the local products are the library's kernels (or a callable
the caller passes), the collectives torch.distributed's (NCCL between GPUs,
gloo between CPU processes). Complex tensors travel as their real views.
"""
from __future__ import annotations

__all__ = ["occupied_ranges", "OccupiedSplit", "gather_block", "sharded_sigma", "sharded_projection"]


def occupied_ranges(nocc, world):
    """Contiguous ranges [i0, i1) of the occupied index for ``world`` ranks, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world must be positive")
    base, extra = divmod(int(nocc), int(world))
    out, i0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((i0, i0 + n))
        i0 += n
    return out


class OccupiedSplit:
    """Which rows of the packed EA vector [X_a (nvir) | X_j,(a<b) (nocc Pv)] a rank holds."""

    def __init__(self, nocc, nvir, world, rank):
        if not 0 <= rank < world:
            raise ValueError("rank outside the group")
        self.nocc, self.nvir, self.world, self.rank = int(nocc), int(nvir), int(world), int(rank)
        self.n1 = self.nvir
        self.pv = self.nvir * (self.nvir - 1) // 2
        self.N = self.n1 + self.nocc * self.pv
        self.ranges = occupied_ranges(self.nocc, self.world)
        self.i0, self.i1 = self.ranges[self.rank]
        self.n_local = self.n1 + (self.i1 - self.i0) * self.pv
        self.max_sat = max(b - a for a, b in self.ranges) * self.pv

    def sat_slice(self, rank=None):
        """Global index range of a rank's satellite rows."""
        a, b = self.ranges[self.rank if rank is None else rank]
        return slice(self.n1 + a * self.pv, self.n1 + b * self.pv)

    def local_of(self, X):
        """This rank's rows [k][n_local] of whole vectors X [k][N] (1p rows, then its satellites)."""
        import torch
        s = self.sat_slice()
        return torch.cat([X[:, :self.n1], X[:, s]], dim=1).contiguous()


def _real(t):
    import torch
    return torch.view_as_real(t) if t.is_complex() else t


def gather_block(split, X_local, group=None):
    """The whole trial block [k][N] on every rank from the ranks' local rows (all-gather)."""
    import torch
    import torch.distributed as dist
    k = X_local.shape[0]
    n1, pv = split.n1, split.pv
    pad = torch.zeros((k, split.max_sat), dtype=X_local.dtype, device=X_local.device)
    pad[:, :X_local.shape[1] - n1] = X_local[:, n1:]
    parts = [torch.empty_like(pad) for _ in range(split.world)]
    dist.all_gather([_real(p) for p in parts], _real(pad), group=group)
    pieces = [X_local[:, :n1]] + [parts[r][:, :(b - a) * pv] for r, (a, b) in enumerate(split.ranges)]
    return torch.cat(pieces, dim=1).contiguous()


def sharded_sigma(split, X_local, share, group=None):
    """S = M X on this rank's rows [k][n_local].

    ``share(X_whole, i0, i1, with_main)`` returns [k][n_local]: the partial 1p
    rows and the complete satellite rows of [i0, i1) (``Context.sigma_share``)."""
    import torch.distributed as dist
    X = gather_block(split, X_local, group)
    S = share(X, split.i0, split.i1, split.rank == 0)
    main = S[:, :split.n1].contiguous()
    dist.all_reduce(_real(main), op=dist.ReduceOp.SUM, group=group)
    S[:, :split.n1] = main
    return S


def sharded_projection(split, V_local, S_local, gram, group=None):
    """G = V^H S over the distributed rows, [m][k] on every rank.

    ``gram(A, B)`` returns sum_n conj(A[a][n]) B[b][n] for row blocks A, B (the
    library's FP64 projection kernel on a GPU); each rank adds its satellite
    rows, rank 0 the 1p rows, and the partial sums are all-reduced."""
    import torch.distributed as dist
    n1 = split.n1
    G = gram(V_local[:, n1:], S_local[:, n1:]).contiguous()
    if split.rank == 0:
        G = G + gram(V_local[:, :n1], S_local[:, :n1])
    G = G.contiguous()
    dist.all_reduce(_real(G), op=dist.ReduceOp.SUM, group=group)
    return G
