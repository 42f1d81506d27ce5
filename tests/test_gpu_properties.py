"""EE ground-to-excited transition densities (adc_transition_density), state
and state-to-state densities of every kind (adc_excited_density,
adc_state_pair_density) and IP/EA spectroscopic amplitudes
(adc_spectroscopic_amplitudes) on the GPU (Sec. 2.2) against the oracle: the closed forms of oracle/properties.py (1e-12 relative, ADC(2) and
ADC(3) contexts) and, on a tiny case, the brute-force ISR transition moments in
determinant space directly (1e-12).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem  # noqa: E402
from oracle import properties as oprop  # noqa: E402
from oracle.integrals import Amplitudes  # noqa: E402
from oracle.isr_series import spectroscopic_series, transition_moments_series  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _vectors(n, k, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    return Y / np.linalg.norm(Y, axis=1, keepdims=True)


@pytest.mark.parametrize("o,v,Q,order,x,seed", [(3, 6, 10, 2, 0.0, 71), (4, 7, 12, 3, 0.5, 72), (2, 5, 8, 3, 1.0, 73)])
def test_transition_density_matches_oracle(gpu, o, v, Q, order, x, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.12, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=order, x=x) as c:
        Y = _vectors(c.N, 2, seed + 1)
        rho = c.transition_density(Y)
        rk = c.excited_density(Y)
    for z in range(2):
        ref = oprop.transition_density(Y[z], p.B, p.eps_occ, p.eps_vir)
        assert np.abs(rho[z] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
        refk = oprop.excited_state_density(Y[z], p.B, p.eps_occ, p.eps_vir)
        assert np.abs(rk[z] - refk).max() < 1e-12 * max(1.0, np.abs(refk).max())


def test_transition_density_matches_isr_series(gpu):
    o, v, Q = 2, 3, 4
    p = make_problem(o, v, Q, seed=1, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    eps = np.concatenate([p.eps_occ, p.eps_vir])
    f, n1, _ = transition_moments_series(eps, p.B, o, nord=3)
    fb = f[0] + f[1] + f[2]
    fb[n1:] = f[0, n1:] + f[1, n1:]
    Y = _vectors(f.shape[1], 1, 2)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=2) as c:
        rho = c.transition_density(Y)[0]
    ref = np.einsum("I,Ipq->pq", Y[0].conj(), fb)
    assert np.abs(rho - ref).max() < 1e-12


def test_transition_density_rejects_ip(gpu):
    p = make_problem(3, 4, 6, seed=3, sigma=0.1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="IP", order=2) as c:
        with pytest.raises(gpu.AdcError) as e:
            c.transition_density(np.zeros((1, c.N), np.complex128))
        assert e.value.code == -6


@pytest.mark.parametrize("kind,o,v,Q,order,x,seed", [("IP", 4, 9, 14, 2, 0.0, 81), ("EA", 4, 9, 14, 3, 0.5, 82),
                                                     ("IP", 12, 40, 60, 3, 1.0, 83), ("EA", 7, 33, 50, 2, 0.0, 84),
                                                     ("IP", 2, 5, 6, 3, 0.5, 85)])
def test_spectroscopic_amplitudes_match_oracle(gpu, kind, o, v, Q, order, x, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.12, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x) as c:
        Y = _vectors(c.N, 3, seed + 1)
        X = c.spectroscopic_amplitudes(Y)
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    for z in range(3):
        ref = oprop.spectroscopic_amplitudes(Y[z], kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
        assert np.abs(X[z] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("kind", ["IP", "EA"])
def test_spectroscopic_amplitudes_match_isr_series(gpu, kind):
    o, v, Q = 2, 3, 4
    p = make_problem(o, v, Q, seed=1, sigma=0.2, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    eps = np.concatenate([p.eps_occ, p.eps_vir])
    f, n1, _ = spectroscopic_series(eps, p.B, o, kind, nord=3)
    fb = f[0] + f[1] + f[2]
    fb[n1:] = f[0, n1:] + f[1, n1:]
    Y = _vectors(f.shape[1], 1, 3)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=2) as c:
        X = c.spectroscopic_amplitudes(Y)[0]
    assert np.abs(X - Y[0].conj() @ fb).max() < 1e-12


def test_spectroscopic_amplitudes_reject_ee(gpu):
    p = make_problem(3, 4, 6, seed=3, sigma=0.1)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=2) as c:
        with pytest.raises(gpu.AdcError) as e:
            c.spectroscopic_amplitudes(np.zeros((1, c.N), np.complex128))
        assert e.value.code == -6


@pytest.mark.parametrize("kind,o,v,Q,order,x,seed", [("IP", 3, 7, 10, 3, 0.5, 91), ("EA", 4, 9, 14, 2, 0.0, 92),
                                                     ("EE", 3, 6, 10, 3, 1.0, 93), ("IP", 10, 37, 50, 2, 0.0, 94),
                                                     ("EA", 6, 29, 40, 3, 0.5, 95)])
def test_state_pair_density_matches_oracle(gpu, kind, o, v, Q, order, x, seed):
    p = make_problem(o, v, Q, seed=seed, sigma=0.12, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x) as c:
        YK = _vectors(c.N, 2, seed + 1)
        YL = _vectors(c.N, 2, seed + 2) * np.array([[1.3], [0.7 - 0.2j]])  # unnormalised ket
        R = c.state_pair_density(YK, YL)
        Rk = c.excited_density(YK)
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    for z in range(2):
        ref = oprop.state_pair_density(YK[z], YL[z], kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
        assert np.abs(R[z] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
        refk = oprop.state_pair_density(YK[z], YK[z], kind, p.B, p.eps_occ, p.eps_vir, amp=amp)
        assert np.abs(Rk[z] - refk).max() < 1e-12 * max(1.0, np.abs(refk).max())
        dn = {"IP": -1, "EA": 1, "EE": 0}[kind]
        assert abs(np.trace(Rk[z]) - (o + dn)) < 1e-11
