"""Pins of the state-specific natural-spinor oracle (Sec. 2.4, Eqs. 31-32).

* The closed-form state density equals <Psi| a+_b a_a |Psi> of the weighted
  configurations evaluated in determinant space (EA: N+1 electrons, EE: N).
* Its trace counts the virtual electrons: 1 per single (EA 1p, EE 1h1p), 2 per
  double (EA 2p1h, EE 2h2p) of a normalised vector.
* Keeping every natural spinor only rotates the virtual space and the
  semicanonical eigenvectors of F are then the canonical spinors up to phase
  and order: ADC(2) and ADC(3) roots are unchanged, the guess carried into the
  new basis overlaps its own root fully, and Eq. 32's correction vanishes.
"""
import numpy as np
import pytest

from synthetic import make_problem
from oracle import ssfns as oss
from oracle.isr_series import FockSpace


def _random_unit(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return y / np.linalg.norm(y)


def _bruteforce_density(kind, y, o, v):
    """<Psi| a+_b a_a |Psi> with |Psi> built from creation/annihilation matrices."""
    fs = FockSpace(o + v)
    ref = np.zeros(fs.dim(o), np.complex128)
    ref[fs.det_index(o, tuple(range(o)))] = 1.0
    nel = o + 1 if kind == "EA" else o
    psi = np.zeros(fs.dim(nel), np.complex128)
    idx = 0
    if kind == "EA":
        for a in range(v):                       # a+_a |Phi>
            psi += y[idx] * (fs.cre(o + a, o) @ ref)
            idx += 1
        for j in range(o):                       # a+_a a+_b a_j |Phi>, a < b
            for a in range(v):
                for b in range(a + 1, v):
                    vec = fs.ann(j, o) @ ref
                    vec = fs.cre(o + b, o - 1) @ vec
                    vec = fs.cre(o + a, o) @ vec
                    psi += y[idx] * vec
                    idx += 1
    else:
        for i in range(o):                       # a+_a a_i |Phi>
            for a in range(v):
                psi += y[idx] * (fs.cre(o + a, o - 1) @ (fs.ann(i, o) @ ref))
                idx += 1
        for i in range(o):                       # a+_a a+_b a_j a_i |Phi>, i < j, a < b
            for j in range(i + 1, o):
                for a in range(v):
                    for b in range(a + 1, v):
                        vec = fs.ann(i, o) @ ref
                        vec = fs.ann(j, o - 1) @ vec
                        vec = fs.cre(o + b, o - 2) @ vec
                        vec = fs.cre(o + a, o - 1) @ vec
                        psi += y[idx] * vec
                        idx += 1
    assert idx == y.size
    D = np.zeros((v, v), np.complex128)
    for a in range(v):
        for b in range(v):
            D[a, b] = np.vdot(psi, fs.excitation(o + b, o + a, nel) @ psi)
    return D


@pytest.mark.parametrize("kind,o,v,seed", [("EA", 2, 3, 1), ("EA", 3, 4, 2), ("EE", 2, 3, 3), ("EE", 3, 3, 4)])
def test_state_density_matches_determinant_space(kind, o, v, seed):
    n = v + o * v * (v - 1) // 2 if kind == "EA" else o * v + (o * (o - 1) // 2) * (v * (v - 1) // 2)
    y = _random_unit(n, seed)
    D = oss.state_density(kind, y, o, v)
    Db = _bruteforce_density(kind, y, o, v)
    assert np.abs(D - Db).max() < 1e-13
    assert np.abs(D - D.conj().T).max() < 1e-14


@pytest.mark.parametrize("kind,o,v,seed", [("EA", 4, 6, 5), ("EE", 3, 5, 6)])
def test_state_density_trace_counts_virtual_electrons(kind, o, v, seed):
    n1 = v if kind == "EA" else o * v
    n = n1 + (o * v * (v - 1) // 2 if kind == "EA" else (o * (o - 1) // 2) * (v * (v - 1) // 2))
    y = _random_unit(n, seed)
    tr = np.trace(oss.state_density(kind, y, o, v)).real
    assert abs(tr - (np.linalg.norm(y[:n1]) ** 2 + 2 * np.linalg.norm(y[n1:]) ** 2)) < 1e-13


@pytest.mark.parametrize("kind,o,v,Q,seed", [("EA", 3, 6, 10, 7), ("EE", 2, 5, 8, 8)])
def test_no_truncation_is_a_rotation(kind, o, v, Q, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    res = oss.ssfns(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir, 3, eta_crit=-1.0)
    w3 = np.linalg.eigvalsh(oss.matrix(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir))
    for k, r in enumerate(res):
        assert r["n_keep"] == v
        assert abs(r["omega2_fns"] - r["omega2_canonical"]) < 1e-10
        assert r["root2"] == k and abs(r["overlap2"] - 1.0) < 1e-10
        assert abs(r["omega_corrected"] - r["omega_fns"]) < 1e-10
        assert np.abs(w3 - r["omega_fns"]).min() < 1e-10
