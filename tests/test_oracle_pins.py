"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
brute-force ISR construction in determinant space (Sec. 2.1, Eqs. 1-7 and 11),
exact FCI energy differences, closed forms and invariants.
"""
import numpy as np
import pytest

from synthetic import make_problem, random_vectors
from oracle import adc
from oracle.integrals import Amplitudes, eri, semicanonical
from oracle.isr_series import (antisym_eri_dense, isr_series, fci_energies,
                               mp1_density_bruteforce, FockSpace, rspt_ground_state)
from oracle import isr_series as isr_mod
from oracle.davidson import lowest_dense, davidson
from oracle.fns import fns_density, fns_basis, transform_cholesky


def _eps(p):
    return np.concatenate([p.eps_occ, p.eps_vir])


# ---------------------------------------------------------------- P1 (Eq. 43)
def test_p1_integrals_reconstruction_and_symmetry():
    o, v, Q = 3, 5, 7
    p = make_problem(o, v, Q, seed=11, sigma=0.3)
    nmo = o + v
    g = antisym_eri_dense(p.B)
    # independent route: Coulomb supermatrix as a Gram matrix of the flattened vectors
    L = p.B.reshape(Q, nmo * nmo)
    C = (L.T @ L).reshape(nmo, nmo, nmo, nmo)  # C[p,r,q,s] = (pr|qs)
    ref = C.transpose(0, 2, 1, 3) - C.transpose(0, 2, 3, 1)
    assert np.abs(g - ref).max() < 1e-15
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() < 1e-15
    assert np.abs(g + g.transpose(0, 1, 3, 2)).max() < 1e-15
    assert np.abs(g.conj() - g.transpose(2, 3, 0, 1)).max() < 1e-15
    # W_(pr),(sq) = sum_Q B_pr conj(B_sq) is Hermitian positive semidefinite
    W = (L.T @ L.conj()).reshape(nmo * nmo, nmo * nmo)
    assert np.linalg.eigvalsh(0.5 * (W + W.conj().T)).min() > -1e-13
    # block accessor agrees with the dense tensor
    blk = eri(p.B, o, "vovo")
    assert np.abs(blk - g[o:, :o, o:, :o]).max() < 1e-15


# ---------------------------------------------------------------- P2
@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_p2_noninteracting_limit(kind):
    o, v = 3, 5
    p = make_problem(o, v, 4, seed=2)
    B0 = np.zeros_like(p.B)
    eo, ev = p.eps_occ, p.eps_vir
    M = adc.explicit_matrix(kind, 3, 1.0, B0, eo, ev)
    w = np.sort(np.linalg.eigvalsh(M))
    if kind == "IP":
        iu, ju = np.triu_indices(o, 1)
        ref = np.concatenate([-eo, (ev[None, :] - eo[iu][:, None] - eo[ju][:, None]).ravel()])
    else:
        iu, ju = np.triu_indices(v, 1)
        ref = np.concatenate([ev, (ev[iu][None, :] + ev[ju][None, :] - eo[:, None]).ravel()])
    assert np.abs(w - np.sort(ref)).max() < 1e-14


@pytest.mark.parametrize("dd", [1, 0])
def test_p2_ee_noninteracting_limit(dd):
    """B = 0: the EE matrix is the orbital-energy differences, eps_a - eps_i
    for the singles and eps_a + eps_b - eps_i - eps_j for the doubles (i<j,
    a<b), at every order and for both doubles-block orders."""
    from oracle import adc_ee
    o, v = 3, 4
    p = make_problem(o, v, 4, seed=2)
    eo, ev = p.eps_occ, p.eps_vir
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    ref = np.sort(np.concatenate([(ev[None, :] - eo[:, None]).ravel(),
                                  ((ev[av] + ev[bv])[None, :] - (eo[io] + eo[jo])[:, None]).ravel()]))
    for order, x in [(2, 0.0), (3, 0.5), (3, 1.0)]:
        M = adc_ee.explicit_matrix(order, x, np.zeros_like(p.B), eo, ev, dd_order=dd)
        assert np.abs(M - np.diag(np.diag(M))).max() == 0.0
        assert np.abs(np.sort(np.linalg.eigvalsh(M)) - ref).max() < 1e-14, (order, x)


# ---------------------------------------------------------------- P3
def test_p3_mp2_energy_matches_rayleigh_schroedinger():
    o, v = 3, 5
    p = make_problem(o, v, 6, seed=4, sigma=0.3)
    eps = _eps(p)
    g = antisym_eri_dense(p.B)
    fs = isr_mod._build_space(eps, g, o)
    sec = isr_mod._Sector(fs, eps, g, o)
    phi = fs.det_index(o, tuple(range(o)))
    _, E = rspt_ground_state(sec, phi, 4)
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    assert abs(E[2] - amp.mp2_energy()) < 1e-14
    assert abs(E[1] + 0.5 * np.einsum("ijij->", g[:o, :o, :o, :o])) < 1e-14
    # third order from the second-order doubles: E3 = 1/4 sum <ij||ab> t2_ij^ab
    e3 = 0.25 * np.einsum("ijab,ijab->", eri(p.B, o, "oovv"), amp.t2d)
    assert abs(E[3] - e3) < 1e-14


# ---------------------------------------------------------------- P5 (strongest)
@pytest.mark.parametrize("kind,o,v,seed", [("IP", 3, 4, 3), ("IP", 4, 3, 7), ("IP", 2, 5, 9),
                                           ("EA", 3, 4, 3), ("EA", 2, 5, 8), ("EA", 4, 3, 10)])
def test_p5_blocks_equal_brute_force_isr_series(kind, o, v, seed):
    p = make_problem(o, v, 6, seed=seed, sigma=0.3)
    r = isr_series(_eps(p), p.B, o, kind, nord=4)
    M, n1 = r["M"], r["n1"]
    bl = adc.Blocks(kind, p.B, p.eps_occ, p.eps_vir)
    scale = np.abs(M).max()
    for n in range(4):
        assert np.abs(M[n][:n1, :n1] - bl.M11[n]).max() < 1e-13 * scale, ("M11", n)
    for n in range(3):
        assert np.abs(M[n][:n1, n1:] - bl.M12[n]).max() < 1e-13 * scale, ("M12", n)
    for n in range(2):
        assert np.abs(M[n][n1:, n1:] - bl.M22[n]).max() < 1e-13 * scale, ("M22", n)
    # the blocks ADC(3) truncates are genuinely nonzero in the ISR (no trivial pass)
    assert np.abs(M[3][:n1, n1:]).max() > 1e-6 and np.abs(M[2][n1:, n1:]).max() > 1e-6


# ---------------------------------------------------------------- P4
@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_p4_error_order_against_fci(kind):
    o, v = 3, 4
    p = make_problem(o, v, 5, seed=21, sigma=0.35)
    eps = _eps(p)
    lams = np.array([0.02, 0.04, 0.08])
    errs = {2: [], 3: [], "x": []}
    for lam in lams:
        E0 = fci_energies(eps, p.B, o, lam, o)[0]
        nel = o - 1 if kind == "IP" else o + 1
        Ex = fci_energies(eps, p.B, o, lam, nel)[0]
        exact = Ex - E0
        Bl = np.sqrt(lam) * p.B
        for key, (order, x) in {2: (2, 0.0), 3: (3, 1.0), "x": (3, 0.5)}.items():
            M = adc.explicit_matrix(kind, order, x, Bl, p.eps_occ, p.eps_vir)
            errs[key].append(abs(np.linalg.eigvalsh(M)[0] - exact))
    s2 = np.polyfit(np.log(lams), np.log(errs[2]), 1)[0]
    s3 = np.polyfit(np.log(lams), np.log(errs[3]), 1)[0]
    assert 2.8 < s2 < 3.2, s2
    assert 3.7 < s3 < 4.3, s3
    ratio = errs["x"][0] / errs[2][0]
    assert abs(ratio - 0.5) < 0.05, ratio


# ---------------------------------------------------------------- P6
@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_p6_hermitian_x_interpolation_and_unit_vectors(kind):
    o, v = 4, 6
    p = make_problem(o, v, 10, seed=13, sigma=0.2)
    bl = adc.Blocks(kind, p.B, p.eps_occ, p.eps_vir)
    M2 = adc.explicit_matrix(kind, 2, 0.7, p.B, p.eps_occ, p.eps_vir, blocks=bl)
    M30 = adc.explicit_matrix(kind, 3, 0.0, p.B, p.eps_occ, p.eps_vir, blocks=bl)
    M31 = adc.explicit_matrix(kind, 3, 1.0, p.B, p.eps_occ, p.eps_vir, blocks=bl)
    Mx = adc.explicit_matrix(kind, 3, 0.3, p.B, p.eps_occ, p.eps_vir, blocks=bl)
    for M in (M2, M31, Mx):
        assert np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()
    assert np.abs(M2 - M30).max() == 0.0
    assert np.abs(Mx - (0.7 * M2 + 0.3 * M31)).max() < 1e-14
    # explicit M times every unit vector equals the matrix-free sigma
    N = M31.shape[0]
    E = np.eye(N, dtype=np.complex128)
    S = adc.sigma_ref(kind, 3, 1.0, p.B, p.eps_occ, p.eps_vir, E)
    assert np.abs(S.T - M31).max() < 1e-14
    S = adc.sigma_ref(kind, 2, 0.0, p.B, p.eps_occ, p.eps_vir, E)
    assert np.abs(S.T - M2).max() < 1e-14
    d = adc.diagonal_ref(kind, 3, 0.3, p.B, p.eps_occ, p.eps_vir)
    assert np.abs(d - np.diag(Mx).real).max() < 1e-14


@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_p6a_unitary_invariance_within_degenerate_groups(kind):
    o, v, Q = 4, 6, 9
    rng = np.random.default_rng(5)
    p = make_problem(o, v, Q, seed=17, sigma=0.2)
    eo = np.repeat(np.sort(rng.uniform(-2, -0.5, o // 2)), 2)
    ev = np.repeat(np.sort(rng.uniform(0.2, 3.0, v // 2)), 2)
    nmo = o + v
    W = np.zeros((nmo, nmo), dtype=np.complex128)
    for g0 in range(0, nmo, 2):
        A = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        q, _ = np.linalg.qr(A)
        W[g0:g0 + 2, g0:g0 + 2] = q
    Br = np.einsum("pi,Qpq,qj->Qij", W.conj(), p.B, W)
    for order, x in [(2, 0.0), (3, 0.5), (3, 1.0)]:
        w0 = np.linalg.eigvalsh(adc.explicit_matrix(kind, order, x, p.B, eo, ev))
        w1 = np.linalg.eigvalsh(adc.explicit_matrix(kind, order, x, Br, eo, ev))
        assert np.abs(w0 - w1).max() < 1e-12


def _random_block_unitary(o, v, rng):
    W = np.zeros((o + v, o + v), dtype=np.complex128)
    for s, n in ((slice(0, o), o), (slice(o, o + v), v)):
        q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        W[s, s] = q
    return W


@pytest.mark.parametrize("kind", ["IP", "EA", "EE"])
def test_p6b_full_fock_blocks_semicanonicalised(kind):
    """Non-degenerate orbital energies, the basis rotated by a random unitary
    within the occupied and within the virtual spinors: the Fock blocks are
    then full. Semicanonicalising them (and rotating B the same way) must give
    back the original eigenvalues; keeping only the diagonal of the rotated
    Fock matrix must not (so the check is not trivially met)."""
    o, v, Q = 3, 5, 7
    rng = np.random.default_rng(23)
    p = make_problem(o, v, Q, seed=29, sigma=0.2)
    U = _random_block_unitary(o, v, rng)
    Br = np.einsum("pi,Qpq,qj->Qij", U.conj(), p.B, U)
    F = U.conj().T @ np.diag(np.concatenate([p.eps_occ, p.eps_vir])) @ U
    eo, ev, Bs = semicanonical(F[:o, :o], F[o:, o:], Br)
    assert np.abs(eo - p.eps_occ).max() < 1e-13 and np.abs(ev - p.eps_vir).max() < 1e-13

    def spectrum(B, e_o, e_v, order, x):
        M = (adc_ee.explicit_matrix(order, x, B, e_o, e_v) if kind == "EE"
             else adc.explicit_matrix(kind, order, x, B, e_o, e_v))
        return np.linalg.eigvalsh(M)

    for order, x in [(2, 0.0), (3, 0.5), (3, 1.0)]:
        w0 = spectrum(p.B, p.eps_occ, p.eps_vir, order, x)
        w1 = spectrum(Bs, eo, ev, order, x)
        assert np.abs(w0 - w1).max() < 1e-12 * max(1.0, np.abs(w0).max()), (order, x)
    wd = spectrum(Br, np.diag(F)[:o].real, np.diag(F)[o:].real, 3, 1.0)
    assert np.abs(spectrum(p.B, p.eps_occ, p.eps_vir, 3, 1.0) - wd).max() > 1e-3


# ---------------------------------------------------------------- P7 (Eq. 25)
def test_p7_mp1_density_matches_brute_force():
    o, v = 3, 5
    p = make_problem(o, v, 6, seed=8, sigma=0.3)
    rho, psi = mp1_density_bruteforce(_eps(p), p.B, o)
    D = fns_density(p.B, p.eps_occ, p.eps_vir)
    assert np.abs(D - rho[o:, o:].T).max() < 1e-15
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir, second_order=False)
    assert np.abs(D - amp.gvv.T).max() < 1e-15
    assert np.abs(D - D.conj().T).max() < 1e-16
    eta = np.linalg.eigvalsh(D)
    assert eta.min() > -1e-16
    norm1 = np.vdot(psi[1], psi[1]).real
    assert abs(np.trace(D).real - 2.0 * norm1) < 1e-15
    assert abs(np.trace(D).real - 0.5 * np.sum(np.abs(amp.t1) ** 2)) < 1e-15


def test_p7_fns_truncation_semicanonical():
    o, v, Q = 4, 12, 20
    p = make_problem(o, v, Q, seed=3, sigma=0.2)
    D = fns_density(p.B, p.eps_occ, p.eps_vir)
    crit = 0.1
    eta, V, n_keep, U, et = fns_basis(D, p.eps_vir, eta_crit=crit)
    assert np.all(np.diff(eta) <= 1e-16)
    assert n_keep == int(np.sum(eta >= crit)) and 0 < n_keep < v
    # retained natural spinors span the eigenvectors with eta >= eta_crit
    assert np.abs(D @ V[:, :n_keep] - V[:, :n_keep] * eta[:n_keep]).max() < 1e-14
    assert np.abs(U.conj().T @ U - np.eye(n_keep)).max() < 1e-13
    F = U.conj().T @ np.diag(p.eps_vir) @ U
    assert np.abs(F - np.diag(et)).max() < 1e-13
    # eta_crit = 0 keeps everything: the transformation is unitary and the
    # spectrum of M is unchanged only if the Fock stays diagonal, which it does
    eta0, V0, nk0, U0, et0 = fns_basis(D, p.eps_vir, eta_crit=-1.0)
    assert nk0 == v
    assert np.abs(np.sort(et0) - np.sort(p.eps_vir)).max() < 1e-13
    Bn = transform_cholesky(p.B, o, U0)
    w0 = np.linalg.eigvalsh(adc.explicit_matrix("IP", 3, 1.0, p.B, p.eps_occ, p.eps_vir))
    w1 = np.linalg.eigvalsh(adc.explicit_matrix("IP", 3, 1.0, Bn, p.eps_occ, et0))
    assert np.abs(w0 - w1).max() < 1e-11


# ---------------------------------------------------------------- P8
@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_p8_davidson_matches_dense(kind):
    o, v = 5, 8
    p = make_problem(o, v, 16, seed=1, sigma=0.15)
    M = adc.explicit_matrix(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir)
    w, _ = lowest_dense(M, 4)
    sig = lambda V: V @ M.T
    d = np.diag(M).real
    wd, Y, rn, it = davidson(sig, d, M.shape[0], 4, tol=1e-9)
    assert np.abs(wd - w).max() < 1e-12
    assert np.all(rn <= 1e-9)
    assert np.abs(Y.conj() @ Y.T - np.eye(4)).max() < 1e-10
    assert np.abs(Y @ M.T - wd[:, None] * Y).max() < 1e-8


# ---------------------------------------------------------------- EE (Eq. 2 manifold)
from oracle import adc_ee  # noqa: E402


@pytest.mark.parametrize("o,v,seed", [(3, 4, 3), (2, 5, 7), (4, 3, 9)])
def test_p5_ee_blocks_equal_brute_force_isr_series(o, v, seed):
    p = make_problem(o, v, 6, seed=seed, sigma=0.3)
    r = isr_series(_eps(p), p.B, o, "EE", nord=4)
    M, n1 = r["M"], r["n1"]
    bl = adc_ee.Blocks(p.B, p.eps_occ, p.eps_vir)
    scale = np.abs(M).max()
    for n in range(4):
        assert np.abs(M[n][:n1, :n1] - bl.MSS[n]).max() < 1e-13 * scale, ("SS", n)
    for n in range(3):
        assert np.abs(M[n][:n1, n1:] - bl.MSD[n]).max() < 1e-13 * scale, ("SD", n)
    for n in range(2):
        assert np.abs(M[n][n1:, n1:] - bl.MDD[n]).max() < 1e-13 * scale, ("DD", n)
    assert np.abs(M[3][:n1, n1:]).max() > 1e-6 and np.abs(M[2][n1:, n1:]).max() > 1e-6


def test_p4_ee_error_order_against_fci():
    o, v = 3, 4
    p = make_problem(o, v, 5, seed=21, sigma=0.35)
    eps = _eps(p)
    lams = np.array([0.02, 0.04, 0.08])
    errs = {2: [], 3: [], "x": [], "dd0": []}
    for lam in lams:
        w = fci_energies(eps, p.B, o, lam, o, nroots=2)
        exact = w[1] - w[0]
        Bl = np.sqrt(lam) * p.B
        for key, (order, x, dd) in {2: (2, 0.0, 1), 3: (3, 1.0, 1), "x": (3, 0.5, 1), "dd0": (3, 1.0, 0)}.items():
            M = adc_ee.explicit_matrix(order, x, Bl, p.eps_occ, p.eps_vir, dd_order=dd)
            errs[key].append(abs(np.linalg.eigvalsh(M)[0] - exact))
    assert 2.8 < np.polyfit(np.log(lams), np.log(errs[2]), 1)[0] < 3.2
    assert 3.7 < np.polyfit(np.log(lams), np.log(errs[3]), 1)[0] < 4.3
    assert abs(errs["x"][0] / errs[2][0] - 0.5) < 0.05
    # ADC(3) with the doubles-doubles block kept at zeroth order: the missing
    # first-order D/D term reaches the singles through two couplings, an
    # O(lambda^3) error, so the slope drops back to 3 (not ADC(2)'s error either)
    assert 2.8 < np.polyfit(np.log(lams), np.log(errs["dd0"]), 1)[0] < 3.2
    assert abs(errs["dd0"][0] / errs[2][0] - 1.0) > 0.2


@pytest.mark.parametrize("order,x,dd", [(3, 1.0, 1), (3, 0.4, 1), (3, 1.0, 0), (2, 0.0, 1)])
def test_p6_ee_sigma_diagonal_hermitian(order, x, dd):
    o, v = 4, 6
    p = make_problem(o, v, 10, seed=13, sigma=0.2)
    M = adc_ee.explicit_matrix(order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd)
    assert np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()
    N = M.shape[0]
    S = adc_ee.sigma_ref(order, x, p.B, p.eps_occ, p.eps_vir, np.eye(N, dtype=np.complex128), dd_order=dd)
    assert np.abs(S.T - M).max() < 1e-13 * np.abs(M).max()
    d = adc_ee.diagonal_ref(order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd)
    assert np.abs(d - np.diag(M).real).max() < 1e-13 * np.abs(M).max()
    if order == 3 and dd == 1 and x == 0.4:
        M0 = adc_ee.explicit_matrix(3, 0.0, p.B, p.eps_occ, p.eps_vir)
        M1 = adc_ee.explicit_matrix(3, 1.0, p.B, p.eps_occ, p.eps_vir)
        assert np.abs(M - (0.6 * M0 + 0.4 * M1)).max() < 1e-14 * np.abs(M).max()


def test_p6a_ee_unitary_invariance_within_degenerate_groups():
    o, v, Q = 4, 6, 9
    rng = np.random.default_rng(5)
    p = make_problem(o, v, Q, seed=17, sigma=0.2)
    eo = np.repeat(np.sort(rng.uniform(-2, -0.5, o // 2)), 2)
    ev = np.repeat(np.sort(rng.uniform(0.2, 3.0, v // 2)), 2)
    nmo = o + v
    W = np.zeros((nmo, nmo), dtype=np.complex128)
    for g0 in range(0, nmo, 2):
        q, _ = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))
        W[g0:g0 + 2, g0:g0 + 2] = q
    Br = np.einsum("pi,Qpq,qj->Qij", W.conj(), p.B, W)
    w0 = np.linalg.eigvalsh(adc_ee.explicit_matrix(3, 0.5, p.B, eo, ev))
    w1 = np.linalg.eigvalsh(adc_ee.explicit_matrix(3, 0.5, Br, eo, ev))
    assert np.abs(w0 - w1).max() < 1e-12


# ---------------------------------------------------------------- P9: eigenvalue derivatives
from oracle import gradients as ograd  # noqa: E402


def _dir(p, seed, dx=0.0):
    rng = np.random.default_rng(seed)
    dB = ograd.random_hermitian_direction(p.B.shape, seed)
    return (dB, rng.standard_normal(p.nocc) * 0.1, rng.standard_normal(p.nvir) * 0.1, dx)


@pytest.mark.parametrize("kind,order,x", [("EE", 3, 0.4), ("EE", 2, 0.0), ("IP", 3, 0.5), ("EA", 3, 1.0)])
def test_p9_hellmann_feynman_equals_eigenvalue_differences(kind, order, x):
    """y^H dM y (central differences of M, h = 1e-5) against central
    differences of the eigenvalues themselves (h = 1e-4): two routes to the
    derivative of a non-degenerate root."""
    o, v = (2, 4) if kind == "EE" else (3, 5)
    p = make_problem(o, v, 6, seed=71, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    D = _dir(p, 5, dx=0.7)
    dw, w, Y = ograd.hf_directional(kind, order, x, p.B, p.eps_occ, p.eps_vir, 3, D)
    assert np.min(np.diff(np.linalg.eigvalsh(ograd.matrix(kind, order, x, p.B, p.eps_occ, p.eps_vir)))[:3]) > 1e-3
    fd = ograd.eig_fd_directional(kind, order, x, p.B, p.eps_occ, p.eps_vir, 3, D)
    assert np.abs(dw - fd).max() < 1e-6 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("kind", ["EE", "EA"])
def test_p9_x_derivative_is_the_adc3_increment(kind):
    """M is linear in x: d omega/dx = y^H (M(x=1) - M(x=0)) y exactly."""
    o, v = (2, 4) if kind == "EE" else (3, 5)
    p = make_problem(o, v, 6, seed=72, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    dw, w, Y = ograd.hf_directional(kind, 3, 0.4, p.B, p.eps_occ, p.eps_vir, 2, (None, None, None, 1.0))
    dM = ograd.matrix(kind, 3, 1.0, p.B, p.eps_occ, p.eps_vir) - ograd.matrix(kind, 3, 0.0, p.B, p.eps_occ,
                                                                               p.eps_vir)
    ref = np.real(np.einsum("rp,pq,rq->r", Y.conj(), dM, Y))
    assert np.abs(dw - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())


def test_p9_noninteracting_orbital_energy_derivatives():
    """B = 0: the lowest EE root is eps_v[0] - eps_o[-1] and the lowest IP root
    is -eps_o[-1], so their derivatives along (deo, dev) are closed forms."""
    p = make_problem(3, 4, 5, seed=73, sigma=0.1, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    B0 = np.zeros_like(p.B)
    rng = np.random.default_rng(3)
    deo, dev = rng.standard_normal(3), rng.standard_normal(4)
    dw, _, _ = ograd.hf_directional("EE", 3, 1.0, B0, p.eps_occ, p.eps_vir, 1, (None, deo, dev, 0.0))
    assert abs(dw[0] - (dev[0] - deo[-1])) < 1e-9
    dw, _, _ = ograd.hf_directional("IP", 3, 1.0, B0, p.eps_occ, p.eps_vir, 1, (None, deo, dev, 0.0))
    assert abs(dw[0] - (-deo[-1])) < 1e-9


def test_p9_complex_gradient_convention():
    """directional() reads gradients as d/dRe + i d/dIm: for f(B) = sum |B|^2
    the gradient 2B predicts the central difference along any direction."""
    rng = np.random.default_rng(4)
    B = rng.standard_normal((2, 3, 3)) + 1j * rng.standard_normal((2, 3, 3))
    dB = ograd.random_hermitian_direction(B.shape, 9)
    h = 1e-6
    fd = (np.sum(np.abs(B + h * dB) ** 2) - np.sum(np.abs(B - h * dB) ** 2)) / (2 * h)
    assert abs(ograd.directional(2 * B, None, None, 0.0, (dB, None, None, 0.0)) - fd) < 1e-7
