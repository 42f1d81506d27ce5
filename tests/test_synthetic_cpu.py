"""The seeded input generators follow the stated recipe.

The generators hold none of the method's arithmetic; these tests pin the
inputs themselves: the Cholesky vectors are Hermitian with circular complex
Gaussian off-diagonal elements of variance sigma^2 and a real diagonal, the
orbital energies are sorted and inside their ranges, the named workloads have
the sizes and method variants of the workloads they stand for, and the
batched workload draws its problems as stated.
"""
import numpy as np
import pytest

from synthetic import (BATCH_CONFIGS, CONFIGS, batch_sizes, make_eri, make_problem, random_hermitian_direction,
                       random_unitary, random_vectors)


def test_cholesky_vectors_hermitian_circular_gaussian():
    sigma = 0.05
    p = make_problem(10, 30, 64, seed=3, sigma=sigma)
    B = p.B
    assert B.shape == (64, 40, 40) and B.dtype == np.complex128
    # exactly Hermitian, real diagonal
    assert np.array_equal(B, np.conj(np.swapaxes(B, 1, 2)))
    d = np.diagonal(B, axis1=1, axis2=2)
    assert np.all(d.imag == 0.0)
    iu, ju = np.triu_indices(40, 1)
    z = B[:, iu, ju].ravel()
    # circular CN(0, sigma^2): E|z|^2 = sigma^2, Re and Im each sigma^2 / 2,
    # uncorrelated, E z^2 = 0 (about 50,000 samples: 3% bounds are > 6 standard errors)
    s2 = sigma ** 2
    assert abs(np.mean(np.abs(z) ** 2) / s2 - 1.0) < 0.03
    assert abs(np.var(z.real) / (s2 / 2) - 1.0) < 0.03
    assert abs(np.var(z.imag) / (s2 / 2) - 1.0) < 0.03
    assert abs(np.mean(z.real * z.imag)) / s2 < 0.03
    assert abs(np.mean(z * z)) / s2 < 0.03
    assert abs(np.mean(z.real)) / sigma < 0.03 and abs(np.mean(z.imag)) / sigma < 0.03
    # diagonal N(0, sigma^2), 2560 samples
    assert abs(np.var(d.real) / s2 - 1.0) < 0.1


def test_orbital_energies_sorted_within_ranges():
    p = make_problem(40, 200, 3, seed=0, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    assert np.all(np.diff(p.eps_occ) >= 0) and np.all(np.diff(p.eps_vir) >= 0)
    assert p.eps_occ.min() >= -3.0 and p.eps_occ.max() <= -0.3
    assert p.eps_vir.min() >= 0.1 and p.eps_vir.max() <= 5.0
    # every occupied level lies below every virtual one (no overlapping energies)
    assert p.eps_occ.max() < p.eps_vir.min()


def test_same_seed_same_inputs():
    a = make_problem(4, 9, 5, seed=11)
    b = make_problem(4, 9, 5, seed=11)
    c = make_problem(4, 9, 5, seed=12)
    assert np.array_equal(a.B, b.B) and np.array_equal(a.eps_occ, b.eps_occ)
    assert not np.array_equal(a.B, c.B)


@pytest.mark.parametrize("name,o,v,q,occ,vir,kind,order,x,nroots", [
    # IP-ADC(3), FP64, 4 roots, Davidson tolerance 1e-8
    ("ip3_o8_v24_q96", 8, 24, 96, (-2.0, -0.5), (0.2, 3.0), "IP", 3, 1.0, 4),
    # EA-ADC(2)+x(3), x = 0.5, 8 roots
    ("ea2x3_o40_v200_q1200", 40, 200, 1200, (-3.0, -0.3), (0.1, 5.0), "EA", 3, 0.5, 8),
    # EE-ADC(3) with the doubles block at the ADC(2) level, 6 roots
    ("ee3_o60_v300_q1800", 60, 300, 1800, (-3.0, -0.3), (0.1, 5.0), "EE", 3, 1.0, 6),
    # EE-ADC(2)+x(3), x = 0.4, 4 roots, gradients
    ("ee2x3_o30_v150_q900", 30, 150, 900, (-3.0, -0.3), (0.1, 5.0), "EE", 3, 0.4, 4),
])
def test_named_workloads(name, o, v, q, occ, vir, kind, order, x, nroots):
    c = CONFIGS[name]
    assert (c["nocc"], c["nvir"], c["naux"]) == (o, v, q)
    assert tuple(c["occ_range"]) == occ and tuple(c["vir_range"]) == vir
    assert (c["kind"], c["order"], c["x"], c["nroots"]) == (kind, order, x, nroots)
    assert c["seed"] == 0 and c.get("sigma", 0.05) == 0.05


def test_ee_adc3_workload_solver_settings():
    c = CONFIGS["ee3_o60_v300_q1800"]
    assert c["dd_order"] == 0 and c["block"] == 12 and c["fns_eta"] == 1e-5
    assert CONFIGS["ip3_o8_v24_q96"]["tol"] == 1e-8


def test_batched_workload_recipe():
    c = BATCH_CONFIGS["batch64_ipea"]
    sizes = batch_sizes("batch64_ipea")
    assert len(sizes) == 64 == c["n"]
    for p, s in enumerate(sizes):
        assert 10 <= s["nocc"] <= 40 and 50 <= s["nvir"] <= 250
        assert s["naux"] == 6 * s["nvir"]
        assert s["kind"] == ("IP" if p % 2 == 0 else "EA") and s["seed"] == p
        assert (s["order"], s["x"]) == (3, 0.5)
    # uneven sizes: the spread the batch scheduler has to balance
    v = [s["nvir"] for s in sizes]
    assert max(v) - min(v) > 100
    assert c["nroots"] == 6


def test_helpers_unit_vectors_unitary_hermitian_direction_psd():
    X = random_vectors(1000, 5, seed=2)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-14)
    U = random_unitary(12, seed=4)
    assert np.abs(U.conj().T @ U - np.eye(12)).max() < 1e-13
    D = random_hermitian_direction((3, 7, 7), seed=5)
    assert np.array_equal(D, np.conj(np.swapaxes(D, 1, 2)))
    assert abs(np.linalg.norm(D) - 1.0) < 1e-14
    V = make_eri(5, 6, seed=1)
    n = 25
    assert V.shape == (n, n) and np.abs(V - V.T).max() < 1e-13
    w = np.linalg.eigvalsh(V)
    assert w.min() > -1e-10 * w.max() and np.sum(w > 1e-10 * w.max()) <= 6
    # symmetric within each index pair: V[(mu nu)][.] = V[(nu mu)][.]
    V4 = V.reshape(5, 5, 5, 5)
    assert np.abs(V4 - V4.transpose(1, 0, 2, 3)).max() < 1e-13
