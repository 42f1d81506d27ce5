"""Pins of the EE transition-density oracle (Sec. 2.2).

* The closed-form transition moments summed into rho_pq = sum_I conj(y_I)
  f_I(pq) equal the brute-force ISR series in determinant space (the
  intermediate states of Eqs. 5-6 and the normalised MP ground state, each a
  perturbation series), singles through second and doubles through first
  order, on every block (vo, ov, oo, vv).
* Each block's leading order separately: the zeroth-order excitation block
  is conj(y), the first-order de-excitation block is sum conj(y_ia) t_ij^ab.
* B = 0: rho is conj(y1) on the excitation block and zero elsewhere.
"""
import numpy as np
import pytest

from synthetic import make_problem
from oracle import adc_ee
from oracle import properties as oprop
from oracle.integrals import Amplitudes
from oracle.isr_series import transition_moments_series


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
