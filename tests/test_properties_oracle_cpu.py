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
from oracle.isr_series import _class_operator, class_indices, isr_series, transition_moments_series


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

