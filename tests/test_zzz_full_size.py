"""Parity at the full sizes of the benchmark workloads, on sampled outputs.

EA-ADC(2)+x(3) at o=40, v=200, Q=1200 (the benchmark's workload) and
EE-ADC(2)+x(3) at o=30, v=150, Q=900: the GPU sigma of one random unit
vector, in FP64 and in the precisions the benchmark times (BF16x3 and the
sliced product), on satellite rows that the oracle computes one at a time
(oracle/rows.py, pinned against the term-by-term sigma in
test_rows_oracle_cpu.py). Tolerances relative to the RMS element of the FP64
sigma: FP64 1e-10, sliced 1e-8 (about 40 significant bits), BF16x3 1e-3
(FP32 accumulation over inner sizes up to 10^5). Runs last: each case holds a
full-size context and takes about a minute of oracle time.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import CONFIGS, config_problem, random_vectors  # noqa: E402
from oracle import rows  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _pair(p, q, n):
    return p * n - p * (p + 1) // 2 + (q - p - 1)


def _check(S64, Sm, Ss, idx, R):
    rms = float(np.sqrt(np.mean(np.abs(S64) ** 2)))
    assert np.abs(S64[:, idx] - R).max() < 1e-10 * rms
    assert np.abs(Ss[:, idx] - R).max() < 1e-8 * rms
    assert np.abs(Sm[:, idx] - R).max() < 1e-3 * rms


def test_ea_full_size_sampled_rows(gpu):
    name = "ea2x3_o40_v200_q1200"
    x = CONFIGS[name]["x"]
    p = config_problem(name)
    o, v = p.nocc, p.nvir
    pv = v * (v - 1) // 2
    X = random_vectors(v + o * pv, 1, seed=21)
    sel = [(3, 17, 150), (37, 0, 199)]
    idx = [v + k * pv + _pair(d, e, v) for k, d, e in sel]
    R = rows.ea_satellite_rows(p.B, p.eps_occ, p.eps_vir, 3, x, X, sel)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EA", order=3, x=x) as c:
        S64 = c.sigma(X, "fp64")
        Sm = c.sigma(X, "bf16x3")
        Ss = c.sigma(X, "sliced")
    _check(S64, Sm, Ss, idx, R)


def test_ee_full_size_sampled_rows(gpu):
    name = "ee2x3_o30_v150_q900"
    x = CONFIGS[name]["x"]
    p = config_problem(name)
    o, v = p.nocc, p.nvir
    n1, po, pv = o * v, o * (o - 1) // 2, v * (v - 1) // 2
    X = random_vectors(n1 + po * pv, 1, seed=22)
    sel = [(2, 17, 33, 140)]
    idx = [n1 + _pair(k, l, o) * pv + _pair(c, d, v) for k, l, c, d in sel]
    R = rows.ee_doubles_rows(p.B, p.eps_occ, p.eps_vir, 3, x, X, sel, dd_order=1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=3, x=x) as c:
        S64 = c.sigma(X, "fp64")
        Sm = c.sigma(X, "bf16x3")
        Ss = c.sigma(X, "sliced")
    _check(S64, Sm, Ss, idx, R)
