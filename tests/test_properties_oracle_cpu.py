"""Pins of the EE transition-density oracle (Sec. 2.2).

* The closed-form transition moments summed into rho_pq = sum_I conj(y_I)
  f_I(pq) equal the brute-force ISR series in determinant space (the
  intermediate states of Eqs. 5-6 and the normalised MP ground state, each a
  perturbation series), singles through second and doubles through first
  order, on every block (vo, ov, oo, vv).
* Each block's leading order separately: the zeroth-order excitation block
  is conj(y), the first-order de-excitation block is sum conj(y_ia) t_ij^ab.
* B = 0: rho is conj(y1) on the excitation block and zero elsewhere.
* The excited-state density (ground state through second order plus the
  configurations weighted by y) equals the same expectation values in
  determinant space; its trace is the electron count and it is Hermitian.
"""
import numpy as np
import pytest

from synthetic import make_problem
from oracle import adc_ee
from oracle import properties as oprop
from oracle.integrals import Amplitudes
from oracle import adc as oadc
from oracle.isr_series import (_class_operator, class_indices, isr_series, spectroscopic_series,
                               transition_moments_series)


def _unit(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return y / np.linalg.norm(y)


@pytest.mark.parametrize("o,v,Q,seed", [(2, 3, 4, 1), (3, 4, 6, 2), (3, 3, 5, 3)])
def test_transition_density_matches_isr_series(o, v, Q, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    eps = np.concatenate([p.eps_occ, p.eps_vir])
    f, n1, _ = transition_moments_series(eps, p.B, o, nord=3)
    y = _unit(f.shape[1], seed)
    fb = f[0] + f[1] + f[2]
    fb[n1:] = f[0, n1:] + f[1, n1:]  # doubles through first order
    rho_b = np.einsum("I,Ipq->pq", y.conj(), fb)
    rho = oprop.transition_density(y, p.B, p.eps_occ, p.eps_vir)
    assert np.abs(rho - rho_b).max() < 1e-14 * max(1.0, np.abs(rho_b).max())
    # leading orders of the two off-diagonal blocks
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    y1c = y[:n1].reshape(o, v).conj()
    r0 = np.einsum("I,Ipq->pq", y.conj(), f[0])
    r1 = np.einsum("I,Ipq->pq", y.conj(), f[1])
    assert np.abs(r0[o:, :o] - y1c.T).max() < 1e-15
    assert np.abs(r1[:o, o:] - np.einsum("ia,ijab->jb", y1c, amp.t1)).max() < 1e-15


def test_transition_density_without_interaction():
    o, v = 3, 4
    p = make_problem(o, v, 5, seed=4, sigma=0.2)
    B0 = np.zeros_like(p.B)
    n1, n2 = adc_ee.dims(o, v)
    y = _unit(n1 + n2, 5)
    rho = oprop.transition_density(y, B0, p.eps_occ, p.eps_vir)
    ref = np.zeros_like(rho)
    ref[o:, :o] = y[:n1].reshape(o, v).conj().T
    assert np.abs(rho - ref).max() < 1e-15


@pytest.mark.parametrize("o,v,Q,seed", [(2, 3, 4, 1), (3, 3, 5, 2), (2, 4, 5, 3)])
def test_excited_state_density_matches_determinant_space(o, v, Q, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    eps = np.concatenate([p.eps_occ, p.eps_vir])
    r = isr_series(eps, p.B, o, "EE", nord=3, want_states=True)
    fs, nel, psi0 = r["fs"], r["nel"], r["psi0"]
    nmo = o + v
    ref = np.zeros(fs.dim(o), np.complex128)
    ref[fs.det_index(o, tuple(range(o)))] = 1.0
    labels = class_indices("EE", o, v)
    Phi = np.array([_class_operator(fs, "EE", c, lab, o) @ ref for c in range(2) for lab in labels[c]])
    y = _unit(Phi.shape[0], seed)
    psi = y @ Phi
    rho_b = np.zeros((nmo, nmo), np.complex128)
    for p_ in range(nmo):
        for q in range(nmo):
            E = fs.excitation(p_, q, nel)
            rho_b[p_, q] = np.vdot(psi, E @ psi) - (1.0 if (p_ == q and p_ < o) else 0.0)
            rho_b[p_, q] += sum(np.vdot(psi0[n], E @ psi0[m]) for n in range(3) for m in range(3 - n))
    rho = oprop.excited_state_density(y, p.B, p.eps_occ, p.eps_vir)
    assert np.abs(rho - rho_b).max() < 1e-13
    assert np.abs(rho - rho.conj().T).max() < 1e-14
    assert abs(np.trace(rho).real - o) < 1e-12



@pytest.mark.parametrize("kind", ["IP", "EA"])
@pytest.mark.parametrize("o,v,Q,seed", [(2, 3, 4, 1), (3, 3, 5, 2), (3, 2, 4, 3)])
def test_spectroscopic_amplitudes_match_isr_series(kind, o, v, Q, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    eps = np.concatenate([p.eps_occ, p.eps_vir])
    f, n1, _ = spectroscopic_series(eps, p.B, o, kind, nord=3)
    y = _unit(f.shape[1], seed + 10)
    fb = f[0] + f[1] + f[2]
    fb[n1:] = f[0, n1:] + f[1, n1:]  # satellites through first order
    x_b = y.conj() @ fb
    x = oprop.spectroscopic_amplitudes(y, kind, p.B, p.eps_occ, p.eps_vir)
    assert np.abs(x - x_b).max() < 1e-14 * max(1.0, np.abs(x_b).max())
    # the orders separately: zeroth is conj(y) on the main orbitals, first is
    # the satellites' t contraction, nothing else
    main = slice(0, o) if kind == "IP" else slice(o, o + v)
    x0 = y.conj() @ f[0]
    ref0 = np.zeros_like(x0)
    ref0[main] = y[:n1].conj()
    assert np.abs(x0 - ref0).max() < 1e-15
    x1 = y.conj() @ f[1]
    assert np.abs(x1[main]).max() < 1e-15
    assert np.abs(x1).max() > 1e-3


@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_spectroscopic_amplitudes_without_interaction(kind):
    o, v = 3, 4
    p = make_problem(o, v, 5, seed=6, sigma=0.2)
    B0 = np.zeros_like(p.B)
    n1, n2 = oadc.dims(kind, o, v)
    y = _unit(n1 + n2, 7)
    x = oprop.spectroscopic_amplitudes(y, kind, B0, p.eps_occ, p.eps_vir)
    ref = np.zeros(o + v, np.complex128)
    ref[slice(0, o) if kind == "IP" else slice(o, o + v)] = y[:n1].conj()
    assert np.abs(x - ref).max() < 1e-15


@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_spectroscopic_strength_sum(kind):
    """Through second order the pole strengths of all states of one class-1
    orbital sum to its occupation (IP: <a+_k a_k>, EA: <a_b a+_b>) of the
    second-order ground state: sum_n |x_p(n)|^2 over a complete set of
    orthonormal y equals (f^H f)_pp, which the series evaluates by brute force."""
    o, v, Q = 2, 3, 4
    p = make_problem(o, v, Q, seed=8, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    n1, n2 = oadc.dims(kind, o, v)
    Y = np.linalg.qr(np.random.default_rng(9).standard_normal((n1 + n2, n1 + n2))
                     + 1j * np.random.default_rng(10).standard_normal((n1 + n2, n1 + n2)))[0].T
    X = np.array([oprop.spectroscopic_amplitudes(y, kind, p.B, p.eps_occ, p.eps_vir) for y in Y])
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    t = amp.t1
    strength = np.sum(np.abs(X) ** 2, axis=0)
    if kind == "IP":
        occ2 = 1.0 - 0.5 * np.einsum("kjab,kjab->k", t.conj(), t).real  # 1 - n_k^(2) hole depletion
        assert np.abs(strength[:o] - occ2).max() < 5e-3 * np.abs(1 - occ2).max() + 1e-12
    else:
        vir2 = 1.0 - 0.5 * np.einsum("ijbc,ijbc->b", t.conj(), t).real
        assert np.abs(strength[o:] - vir2).max() < 5e-3 * np.abs(1 - vir2).max() + 1e-12


def _ground_series_density(eps, B, o, nord=3):
    """sum_{n+m<nord} <psi0^(n)| a+_p a_q |psi0^(m)> of the normalised MP ground state."""
    from oracle.isr_series import (_Sector, _build_space, _inv_sqrt, _scombine, _sdot, antisym_eri_dense,
                                   rspt_ground_state)
    g = antisym_eri_dense(B)
    fs = _build_space(eps, g, o)
    secN = _Sector(fs, eps, g, o)
    psi, _ = rspt_ground_state(secN, fs.det_index(o, tuple(range(o))), nord)
    psi0 = _scombine(psi[:, None, :], _inv_sqrt(_sdot(psi[:, None, :], psi[:, None, :])))[:, 0, :]
    nmo = eps.shape[0]
    r = np.zeros((nmo, nmo), np.complex128)
    for p_ in range(nmo):
        for q in range(nmo):
            E = fs.excitation(p_, q, o)
            r[p_, q] = sum(np.vdot(psi0[n], E @ psi0[m]) for n in range(nord) for m in range(nord - n))
    return r, fs


@pytest.mark.parametrize("kind", ["IP", "EA", "EE"])
@pytest.mark.parametrize("o,v,Q,seed", [(2, 3, 4, 11), (3, 3, 5, 12)])
def test_state_pair_density_matches_determinant_space(kind, o, v, Q, seed):
    """<Psi_K|a+_p a_q|Psi_L> with Psi = the configurations weighted by y in the
    target sector, minus (y_K^H y_L) times the reference density, plus
    (y_K^H y_L) times the ground-state density series: every block, K != L."""
    p = make_problem(o, v, Q, seed=seed, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    eps = np.concatenate([p.eps_occ, p.eps_vir])
    rho0, fs = _ground_series_density(eps, p.B, o)
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    assert np.abs(oprop.ground_state_density(amp) - rho0).max() < 1e-13
    ref = np.zeros(fs.dim(o), np.complex128)
    ref[fs.det_index(o, tuple(range(o)))] = 1.0
    labels = class_indices(kind, o, v)
    Phi = np.array([_class_operator(fs, kind, c, lab, o) @ ref for c in range(2) for lab in labels[c]])
    nel = {"IP": o - 1, "EA": o + 1, "EE": o}[kind]
    rng = np.random.default_rng(seed)
    yK = rng.standard_normal(Phi.shape[0]) + 1j * rng.standard_normal(Phi.shape[0])
    yL = rng.standard_normal(Phi.shape[0]) + 1j * rng.standard_normal(Phi.shape[0])
    pK, pL = yK @ Phi, yL @ Phi
    s = np.vdot(yK, yL)
    nmo = o + v
    rho_b = np.zeros((nmo, nmo), np.complex128)
    for p_ in range(nmo):
        for q in range(nmo):
            E = fs.excitation(p_, q, nel)
            rho_b[p_, q] = np.vdot(pK, E @ pL) - (s if (p_ == q and p_ < o) else 0.0)
    rho_b += s * rho0
    rho = oprop.state_pair_density(yK, yL, kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
    assert np.abs(rho - rho_b).max() < 1e-13 * max(1.0, np.abs(rho_b).max())
    # rho^LK = (rho^KL)^H
    rho_lk = oprop.state_pair_density(yL, yK, kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
    assert np.abs(rho_lk - rho.conj().T).max() < 1e-14 * np.abs(rho).max()


@pytest.mark.parametrize("kind,dn", [("IP", -1), ("EA", 1), ("EE", 0)])
def test_state_pair_density_traces(kind, dn):
    """Normalised state: trace = electrons of the target sector, Hermitian,
    equal to the EE excited-state density for EE; orthogonal pair: trace 0."""
    o, v, Q = 3, 5, 7
    p = make_problem(o, v, Q, seed=21, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    n = o * v + adc_ee.dims(o, v)[1] if kind == "EE" else sum(oadc.dims(kind, o, v))
    Yq = np.linalg.qr(np.random.default_rng(22).standard_normal((n, 2))
                      + 1j * np.random.default_rng(23).standard_normal((n, 2)))[0].T
    r = oprop.state_pair_density(Yq[0], Yq[0], kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
    assert abs(np.trace(r) - (o + dn)) < 1e-12
    assert np.abs(r - r.conj().T).max() < 1e-14
    r01 = oprop.state_pair_density(Yq[0], Yq[1], kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
    assert abs(np.trace(r01)) < 1e-12
    if kind == "EE":
        assert np.abs(r - oprop.excited_state_density(Yq[0], p.B, p.eps_occ, p.eps_vir, amp=amp)).max() < 1e-15
