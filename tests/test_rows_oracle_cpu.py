"""Pins of the row oracles (oracle/rows.py), which compute single rows of
S = M X at sizes where the dense oracle cannot: every row equals the same
row of the term-by-term sigma (adc.sigma_ref, adc_ee.sigma_ref; Sec. 2.1) on
small problems, for ADC(2), ADC(2)+x(3), ADC(3) and both EE doubles-block
orders, so the full-size sampled parity tests and the CPU baseline use rows
that are pinned to the oracle's definition."""
import numpy as np
import pytest

from synthetic import make_problem, random_vectors
from oracle import adc, adc_ee, rows


def _pair(p, q, n):
    return p * n - p * (p + 1) // 2 + (q - p - 1)


@pytest.mark.parametrize("order,x", [(2, 0.0), (3, 1.0), (3, 0.5)])
def test_ea_rows_equal_sigma(order, x):
    o, v, Q = 3, 6, 9
    p = make_problem(o, v, Q, seed=41, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    n1, n2 = adc.dims("EA", o, v)
    X = random_vectors(n1 + n2, 2, seed=42)
    S = adc.sigma_ref("EA", order, x, p.B, p.eps_occ, p.eps_vir, X)
    sel = [(0, 0, 1), (2, 3, 5), (1, 0, 4), (2, 1, 2)]
    R = rows.ea_satellite_rows(p.B, p.eps_occ, p.eps_vir, order, x, X, sel)
    idx = [n1 + k * (v * (v - 1) // 2) + _pair(d, e, v) for k, d, e in sel]
    assert np.abs(R - S[:, idx]).max() < 1e-13 * max(1.0, np.abs(S).max())


@pytest.mark.parametrize("order,x", [(2, 0.0), (3, 1.0), (3, 0.5)])
def test_ip_rows_equal_sigma(order, x):
    o, v, Q = 4, 5, 9
    p = make_problem(o, v, Q, seed=43, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    n1, n2 = adc.dims("IP", o, v)
    X = random_vectors(n1 + n2, 2, seed=44)
    S = adc.sigma_ref("IP", order, x, p.B, p.eps_occ, p.eps_vir, X)
    sel = [(0, 1, 0), (2, 3, 4), (1, 3, 2), (0, 2, 1)]
    R = rows.ip_satellite_rows(p.B, p.eps_occ, p.eps_vir, order, x, X, sel)
    idx = [n1 + _pair(i, j, o) * v + a for i, j, a in sel]
    assert np.abs(R - S[:, idx]).max() < 1e-13 * max(1.0, np.abs(S).max())


@pytest.mark.parametrize("order,x,dd", [(2, 0.0, 1), (3, 1.0, 1), (3, 0.7, 0), (3, 0.4, 1)])
def test_ee_rows_equal_sigma(order, x, dd):
    o, v, Q = 3, 5, 8
    p = make_problem(o, v, Q, seed=45, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    n1, n2 = adc_ee.dims(o, v)
    X = random_vectors(n1 + n2, 2, seed=46)
    S = adc_ee.sigma_ref(order, x, p.B, p.eps_occ, p.eps_vir, X, dd_order=dd)
    sel = [(0, 1, 0, 1), (1, 2, 2, 4), (0, 2, 1, 3)]
    R = rows.ee_doubles_rows(p.B, p.eps_occ, p.eps_vir, order, x, X, sel, dd_order=dd)
    pv = v * (v - 1) // 2
    idx = [n1 + _pair(k, l, o) * pv + _pair(c, d, v) for k, l, c, d in sel]
    assert np.abs(R - S[:, idx]).max() < 1e-13 * max(1.0, np.abs(S).max())


@pytest.mark.parametrize("kind", ["EA", "IP"])
@pytest.mark.parametrize("order,x", [(2, 0.0), (3, 1.0), (3, 0.5)])
def test_main_rows_equal_sigma(kind, order, x):
    """The 1p (EA) / 1h (IP) rows of the full-size row oracle, built from the
    per-index ground state of rows.main_rows_ground, equal the term-by-term
    sigma."""
    o, v, Q = (3, 6, 9) if kind == "EA" else (4, 5, 9)
    p = make_problem(o, v, Q, seed=47, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    n1, n2 = adc.dims(kind, o, v)
    X = random_vectors(n1 + n2, 2, seed=48)
    S = adc.sigma_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, X)
    g = rows.main_rows_ground(p.B, p.eps_occ, p.eps_vir)
    fn = rows.ea_main_rows if kind == "EA" else rows.ip_main_rows
    sel = list(range(n1))
    R = fn(p.B, p.eps_occ, p.eps_vir, order, x, X, sel, ground=g)
    assert np.abs(R - S[:, sel]).max() < 1e-13 * max(1.0, np.abs(S).max())


def test_main_rows_ground_equals_amplitudes():
    """The index-by-index ground state equals integrals.Amplitudes."""
    from oracle.integrals import Amplitudes
    p = make_problem(3, 5, 8, seed=49, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    g = rows.main_rows_ground(p.B, p.eps_occ, p.eps_vir)
    a = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    for key, ref in (("t1", a.t1), ("t2s", a.t2s), ("t2d", a.t2d), ("gvv", a.gvv), ("hoo", a.hoo)):
        assert np.abs(g[key] - ref).max() < 1e-14 * max(1.0, np.abs(ref).max()), key
