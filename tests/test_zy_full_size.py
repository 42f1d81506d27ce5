"""Parity at the full sizes of the benchmark workloads, on sampled outputs.

The GPU sigma of one random unit vector, in FP64 and in the precisions the
benchmark times (BF16x3 and the sliced product), against rows of S = M X
that the oracle computes one at a time (oracle/rows.py, pinned against the
term-by-term sigma in test_rows_oracle_cpu.py), at least eight rows of each
class per case:
* EA-ADC(2)+x(3) at o=40, v=200, Q=1200 (the benchmark's workload): 1p rows
  (main block to third order plus the coupling of the satellites) and 2p1h
  satellite rows;
* IP-ADC(2)+x(3), x = 0.5, on the same inputs: 1h rows and 2h1p rows;
* EE-ADC(2)+x(3) at o=30, v=150, Q=900: doubles rows.
Tolerances relative to the RMS element of the FP64 sigma: FP64 1e-10, sliced
1e-8 (about 40 significant bits), BF16x3 1e-3 (FP32 accumulation over inner
sizes up to 10^5). The main rows share one ground state (second-order
amplitudes built index by index, about two minutes on the host cores); the
other rows run in parallel processes. Runs last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import CONFIGS, config_problem, random_vectors  # noqa: E402
from oracle import rows  # noqa: E402

EA = "ea2x3_o40_v200_q1200"


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


@pytest.fixture(scope="module")
def ea_inputs():
    p = config_problem(EA)
    return p, rows.main_rows_ground(p.B, p.eps_occ, p.eps_vir)


def _pair(p, q, n):
    return p * n - p * (p + 1) // 2 + (q - p - 1)


def _check(S64, Sm, Ss, idx, R, what):
    rms = float(np.sqrt(np.mean(np.abs(S64) ** 2)))
    assert np.abs(S64[:, idx] - R).max() < 1e-10 * rms, (what, "fp64")
    assert np.abs(Ss[:, idx] - R).max() < 1e-8 * rms, (what, "sliced")
    assert np.abs(Sm[:, idx] - R).max() < 1e-3 * rms, (what, "bf16x3")


def _gpu_sigmas(gpu, p, kind, x, X):
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=x) as c:
        return c.sigma(X, "fp64"), c.sigma(X, "bf16x3"), c.sigma(X, "sliced")


def test_ea_full_size_sampled_rows(gpu, ea_inputs):
    from conftest import oracle_rows_pool
    p, g = ea_inputs
    x = CONFIGS[EA]["x"]
    o, v = p.nocc, p.nvir
    pv = v * (v - 1) // 2
    X = random_vectors(v + o * pv, 1, seed=21)
    main = [0, 3, 57, 99, 100, 150, 198, 199]
    sat = [(3, 17, 150), (37, 0, 199), (0, 1, 2), (39, 197, 198), (12, 45, 46), (20, 0, 100), (5, 120, 121),
           (31, 77, 190)]
    Rm = rows.ea_main_rows(p.B, p.eps_occ, p.eps_vir, 3, x, X, main, ground=g)
    Rs = oracle_rows_pool(EA, "EA", 3, x, X, sat)
    S64, Sm, Ss = _gpu_sigmas(gpu, p, "EA", x, X)
    _check(S64, Sm, Ss, main, Rm, "1p rows")
    _check(S64, Sm, Ss, [v + k * pv + _pair(d, e, v) for k, d, e in sat], Rs, "2p1h rows")


def test_ip_full_size_sampled_rows(gpu, ea_inputs):
    from conftest import oracle_rows_pool
    p, g = ea_inputs
    x = 0.5
    o, v = p.nocc, p.nvir
    po = o * (o - 1) // 2
    X = random_vectors(o + po * v, 1, seed=23)
    main = [0, 1, 7, 19, 20, 33, 38, 39]
    sat = [(0, 1, 0), (38, 39, 199), (3, 17, 150), (10, 30, 99), (0, 39, 5), (22, 23, 180), (5, 6, 64),
           (14, 27, 133)]
    Rm = rows.ip_main_rows(p.B, p.eps_occ, p.eps_vir, 3, x, X, main, ground=g)
    Rs = oracle_rows_pool(EA, "IP", 3, x, X, sat)
    S64, Sm, Ss = _gpu_sigmas(gpu, p, "IP", x, X)
    _check(S64, Sm, Ss, main, Rm, "1h rows")
    _check(S64, Sm, Ss, [o + _pair(i, j, o) * v + a for i, j, a in sat], Rs, "2h1p rows")


def test_ee_full_size_sampled_rows(gpu):
    from conftest import oracle_rows_pool
    name = "ee2x3_o30_v150_q900"
    x = CONFIGS[name]["x"]
    p = config_problem(name)
    o, v = p.nocc, p.nvir
    n1, po, pv = o * v, o * (o - 1) // 2, v * (v - 1) // 2
    X = random_vectors(n1 + po * pv, 1, seed=22)
    sel = [(2, 17, 33, 140), (0, 1, 0, 1), (28, 29, 148, 149), (5, 20, 10, 90), (13, 14, 70, 71),
           (0, 29, 0, 149), (9, 21, 44, 120), (17, 26, 3, 60)]
    R = oracle_rows_pool(name, "EE", 3, x, X, sel, dd_order=1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=x) as c:
        S64 = c.sigma(X, "fp64")
        Sm = c.sigma(X, "bf16x3")
        Ss = c.sigma(X, "sliced")
    _check(S64, Sm, Ss, [n1 + _pair(k, l, o) * pv + _pair(c, d, v) for k, l, c, d in sel], R, "doubles rows")
