"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module draws random numbers only. It holds none of the method's
arithmetic (no integrals, amplitudes or matrix elements), so the CPU oracle
and the CUDA path can both consume its arrays without sharing any code.

Draw recipe (stated once, used everywhere):

* ``rng = numpy.random.default_rng(seed)``.
* ``eps_occ``: ``nocc`` draws ``uniform(lo_o, hi_o)``, sorted ascending.
* ``eps_vir``: ``nvir`` draws ``uniform(lo_v, hi_v)``, sorted ascending.
* ``B``: ``[naux][nmo][nmo]`` complex, occupied spinors first. All diagonal
  elements are drawn first as one ``standard_normal((naux, nmo))`` block,
  scaled by ``sigma`` (real). The strict upper triangle is then drawn as one
  ``standard_normal((naux, nmo*(nmo-1)/2, 2))`` block (row-major pair order),
  scaled by ``sigma/sqrt(2)`` for the real and imaginary parts, i.e. a
  circular complex Gaussian of variance ``sigma**2``. The lower triangle is
  the complex conjugate, so every ``B[Q]`` is Hermitian, as the Cholesky
  vectors of a Hermitian two-electron integral matrix in a spinor basis are.
* Trial vectors: ``standard_normal`` real and imaginary planes, each
  vector normalised to unit 2-norm.
"""
from __future__ import annotations

import numpy as np

__all__ = ["Problem", "make_problem", "random_vectors", "CONFIGS", "config_problem", "batch_sizes",
           "batch_problems", "BATCH_CONFIGS"]


class Problem:
    """Container for one synthetic input set (all arrays host numpy)."""

    def __init__(self, B, eps_occ, eps_vir, kind, order, x, seed, name=""):
        self.B = B
        self.eps_occ = eps_occ
        self.eps_vir = eps_vir
        self.kind = kind
        self.order = order
        self.x = x
        self.seed = seed
        self.name = name

    @property
    def nocc(self):
        return int(self.eps_occ.shape[0])

    @property
    def nvir(self):
        return int(self.eps_vir.shape[0])

    @property
    def naux(self):
        return int(self.B.shape[0])

    def __repr__(self):
        return (f"Problem({self.name!r}, kind={self.kind}, order={self.order}, x={self.x}, "
                f"nocc={self.nocc}, nvir={self.nvir}, naux={self.naux}, seed={self.seed})")


def make_problem(nocc, nvir, naux, seed=0, sigma=0.05, occ_range=(-2.0, -0.5),
                 vir_range=(0.2, 3.0), kind="IP", order=3, x=1.0, name="",
                 dtype=np.complex128):
    rng = np.random.default_rng(seed)
    eps_occ = np.sort(rng.uniform(occ_range[0], occ_range[1], nocc))
    eps_vir = np.sort(rng.uniform(vir_range[0], vir_range[1], nvir))
    nmo = nocc + nvir
    B = np.empty((naux, nmo, nmo), dtype=dtype)
    diag = rng.standard_normal((naux, nmo)) * sigma
    iu, ju = np.triu_indices(nmo, k=1)
    off = rng.standard_normal((naux, iu.shape[0], 2)) * (sigma / np.sqrt(2.0))
    offc = off[..., 0] + 1j * off[..., 1]
    del off
    B[:, iu, ju] = offc
    B[:, ju, iu] = np.conj(offc)
    del offc
    di = np.arange(nmo)
    B[:, di, di] = diag
    return Problem(B, eps_occ, eps_vir, kind, order, x, seed, name)


def make_eri(nao, rank, seed=0, decay=0.7):
    """Synthetic AO two-electron integrals as the PSD matrix V[(mu nu)][(kappa lambda)].

    V = sum_g w_g G_g G_g^T with real symmetric G_g (mu <-> nu), weights
    w_g = decay^g: real, symmetric in each index pair and between the pairs,
    positive semidefinite of rank <= `rank`, with the decaying spectrum a
    Cholesky decomposition of integrals meets. Returns V [nao*nao][nao*nao].
    """
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((rank, nao, nao))
    G = 0.5 * (G + G.transpose(0, 2, 1))
    w = decay ** np.arange(rank)
    Gf = G.reshape(rank, nao * nao)
    return np.ascontiguousarray((Gf.T * w) @ Gf)


def random_unitary(n, seed=0):
    """Haar-random complex unitary n x n (QR of a complex Gaussian, phases fixed)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Qm, R = np.linalg.qr(A)
    return Qm * (np.diag(R) / np.abs(np.diag(R)))[None, :]


def random_vectors(n, k, seed=1):
    """``k`` complex unit vectors of length ``n`` as a ``[k][n]`` complex128 array."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    return X


# The five named workloads (sizes, ranges, method variant). Names describe
# what each is; the arrays are drawn by make_problem with the stated seed.
CONFIGS = {
    "ip3_o8_v24_q96": dict(nocc=8, nvir=24, naux=96, seed=0, occ_range=(-2.0, -0.5),
                           vir_range=(0.2, 3.0), kind="IP", order=3, x=1.0, nroots=4, tol=1e-8),
    "ea2x3_o40_v200_q1200": dict(nocc=40, nvir=200, naux=1200, seed=0, occ_range=(-3.0, -0.3),
                                 vir_range=(0.1, 5.0), kind="EA", order=3, x=0.5, nroots=8, tol=1e-6),
    # EE-ADC(3) with the doubles block at the ADC(2) level, block Davidson of 12,
    # the FNS virtual density truncated at occupation 1e-5
    "ee3_o60_v300_q1800": dict(nocc=60, nvir=300, naux=1800, seed=0, occ_range=(-3.0, -0.3),
                               vir_range=(0.1, 5.0), kind="EE", order=3, x=1.0, nroots=6, tol=1e-6,
                               dd_order=0, block=12, fns_eta=1e-5, setup="sliced", fp64_davidson=False,
                               gradient=False),
    "ee2x3_o30_v150_q900": dict(nocc=30, nvir=150, naux=900, seed=0, occ_range=(-3.0, -0.3),
                                vir_range=(0.1, 5.0), kind="EE", order=3, x=0.4, nroots=4, tol=1e-8),
    # a smaller case of the same family, for quick runs of the same measurement
    "ee2x3_o12_v60_q360": dict(nocc=12, nvir=60, naux=360, seed=0, occ_range=(-3.0, -0.3),
                               vir_range=(0.1, 5.0), kind="EE", order=3, x=0.4, nroots=4, tol=1e-8),
    # stretch shape: the EA workload with twice the virtual spinors, whose packed
    # <ab||cd> (102 GB) is past the stored form, so the ladder is integral-direct
    "ea2x3_o40_v400_q2000": dict(nocc=40, nvir=400, naux=2000, seed=0, occ_range=(-3.0, -0.3),
                                 vir_range=(0.1, 5.0), kind="EA", order=3, x=0.5, nroots=8, tol=1e-6,
                                 fp64_davidson=False),
}


# solver settings of a config (not inputs of make_problem)
SOLVER_KEYS = ("nroots", "tol", "dd_order", "block", "fns_eta", "setup", "fp64_davidson", "gradient")


def config_problem(name):
    c = {k: val for k, val in CONFIGS[name].items() if k not in SOLVER_KEYS}
    return make_problem(name=name, **c)


# Batched IP/EA workload: problem p draws nocc uniform in [10, 40] and nvir
# uniform in [50, 250] (integers, both ends included) from default_rng(p), takes
# naux = 6 nvir, is IP for even p and EA for odd p, ADC(2)+x(3) with x = 0.5,
# and its inputs come from make_problem(..., seed=p) with the wide energy ranges.
BATCH_CONFIGS = {
    "batch64_ipea": dict(n=64, occ=(10, 40), vir=(50, 250), aux_per_vir=6, order=3, x=0.5, nroots=6, tol=1e-5,
                         occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0)),
}


def batch_sizes(name="batch64_ipea", n=None):
    """Sizes of the batched workload without the arrays: list of dicts."""
    c = BATCH_CONFIGS[name]
    out = []
    for p in range(c["n"] if n is None else n):
        rng = np.random.default_rng(p)
        o = int(rng.integers(c["occ"][0], c["occ"][1] + 1))
        v = int(rng.integers(c["vir"][0], c["vir"][1] + 1))
        out.append(dict(kind="IP" if p % 2 == 0 else "EA", nocc=o, nvir=v, naux=c["aux_per_vir"] * v,
                        order=c["order"], x=c["x"], seed=p))
    return out


def batch_problems(name="batch64_ipea", n=None, select=None):
    """The problems of the batched workload (host arrays), optionally a subset of indices."""
    c = BATCH_CONFIGS[name]
    sizes = batch_sizes(name, n)
    idx = range(len(sizes)) if select is None else select
    return [make_problem(sizes[i]["nocc"], sizes[i]["nvir"], sizes[i]["naux"], seed=sizes[i]["seed"],
                         occ_range=c["occ_range"], vir_range=c["vir_range"], kind=sizes[i]["kind"],
                         order=c["order"], x=c["x"], name=f"{name}[{i}]") for i in idx]


def random_hermitian_direction(shape, seed):
    """Random dB [Q][n][n] with every dB[Q] Hermitian and unit Frobenius norm (a
    perturbation direction of Cholesky vectors)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    A = 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))
    return np.ascontiguousarray(A / np.linalg.norm(A))

