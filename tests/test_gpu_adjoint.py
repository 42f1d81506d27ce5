"""Adjoint of the IP-, EA- and EE-ADC matrices (adc_sigma_adjoint) and the differentiable
roots (torch.autograd): gradients with respect to B, the orbital energies and
x against the oracle's Hellmann-Feynman derivative y^H dM y (explicit matrix,
central differences, h = 1e-5) along random directions, and against central
differences of the GPU's own FP64 eigenvalues.

Tolerance 1e-7 relative for the adjoint against the oracle (the central
difference of M has an O(h^2) = 1e-10 error, the adjoint is FP64 throughout),
1e-6 relative against eigenvalue differences (Davidson residual 1e-10, step
1e-5: the eigenvalue error tol^2/gap, divided by 2h, stays below 1e-9).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem  # noqa: E402
from oracle import gradients as ograd  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


CASES = [
    (2, 4, 6, 3, 0.4, 1, 81),   # ADC(2)+x(3)
    (3, 5, 8, 3, 1.0, 0, 82),   # ADC(3), doubles block at ADC(2) level
    (2, 5, 7, 2, 0.0, 1, 83),   # ADC(2)
    (3, 4, 6, 3, 0.0, 1, 84),   # x = 0 at third order: d/dx still non-zero
    (3, 6, 9, 3, 1.0, 1, 85),   # full ADC(3)
]


def _problem(o, v, Q, seed):
    return make_problem(o, v, Q, seed=seed, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))


@pytest.mark.parametrize("o,v,Q,order,x,dd,seed", CASES)
def test_adjoint_matches_hellmann_feynman(gpu, o, v, Q, order, x, dd, seed):
    p = _problem(o, v, Q, seed)
    nr = 3
    M = ograd.matrix("EE", order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd)
    w, V = np.linalg.eigh(M)
    assert np.diff(w[:nr + 1]).min() > 1e-4
    Y = np.ascontiguousarray(V[:, :nr].T)
    g = np.random.default_rng(seed).standard_normal(nr)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=order, x=x, dd_order=dd) as c:
        gB, geo, gev, gx = c.sigma_adjoint(Y, g)
    rng = np.random.default_rng(seed + 1)
    dB = ograd.random_hermitian_direction(p.B.shape, seed + 2)
    deo, dev = rng.standard_normal(o), rng.standard_normal(v)
    dirs = {"B": (dB, None, None, 0.0), "eps_occ": (None, deo, None, 0.0), "eps_vir": (None, None, dev, 0.0),
            "x": (None, None, None, 1.0), "all": (dB, deo, dev, 0.5)}
    for name, D in dirs.items():
        dw, _, _ = ograd.hf_directional("EE", order, x, p.B, p.eps_occ, p.eps_vir, nr, D, dd_order=dd, Y=Y)
        ref = float(np.dot(g, dw))
        pred = ograd.directional(gB, geo, gev, gx, D)
        assert abs(pred - ref) < 1e-7 * max(1.0, abs(ref)), (name, pred, ref)
    if order == 2:
        assert gx == 0.0


CASES_IPEA = [
    ("IP", 4, 6, 8, 3, 0.5, 91),   # ADC(2)+x(3)
    ("EA", 3, 6, 8, 3, 0.5, 92),
    ("IP", 4, 5, 6, 2, 0.0, 93),   # ADC(2)
    ("EA", 3, 5, 7, 2, 0.0, 94),
    ("EA", 4, 5, 8, 3, 0.0, 95),   # x = 0 at third order: d/dx still non-zero
    ("IP", 5, 6, 8, 3, 1.0, 96),   # ADC(3)
    ("EA", 3, 7, 9, 3, 1.0, 97),
]


@pytest.mark.parametrize("kind,o,v,Q,order,x,seed", CASES_IPEA)
def test_adjoint_ipea_matches_hellmann_feynman(gpu, kind, o, v, Q, order, x, seed):
    p = _problem(o, v, Q, seed)
    nr = 3
    M = ograd.matrix(kind, order, x, p.B, p.eps_occ, p.eps_vir)
    w, V = np.linalg.eigh(M)
    assert np.diff(w[:nr + 1]).min() > 1e-4
    Y = np.ascontiguousarray(V[:, :nr].T)
    g = np.random.default_rng(seed).standard_normal(nr)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=order, x=x) as c:
        gB, geo, gev, gx = c.sigma_adjoint(Y, g)
    rng = np.random.default_rng(seed + 1)
    dB = ograd.random_hermitian_direction(p.B.shape, seed + 2)
    deo, dev = rng.standard_normal(o), rng.standard_normal(v)
    dirs = {"B": (dB, None, None, 0.0), "eps_occ": (None, deo, None, 0.0), "eps_vir": (None, None, dev, 0.0),
            "x": (None, None, None, 1.0), "all": (dB, deo, dev, 0.5)}
    for name, D in dirs.items():
        dw, _, _ = ograd.hf_directional(kind, order, x, p.B, p.eps_occ, p.eps_vir, nr, D, Y=Y)
        ref = float(np.dot(g, dw))
        pred = ograd.directional(gB, geo, gev, gx, D)
        assert abs(pred - ref) < 1e-7 * max(1.0, abs(ref)), (name, pred, ref)
    if order == 2:
        assert gx == 0.0


def test_adjoint_rejects_bad_weights(gpu):
    p = _problem(3, 5, 6, 86)
    for kind in ("IP", "EE"):
        with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=2) as c:
            Y = np.zeros((1, c.N), np.complex128)
            Y[0, 0] = 1.0
            with pytest.raises(gpu.AdcError) as e:
                c.sigma_adjoint(Y, [np.nan])
            assert e.value.code == -1


@pytest.mark.parametrize("kind,o,v,Q,seed", [("EE", 4, 10, 16, 87), ("EA", 5, 12, 20, 88), ("IP", 8, 10, 20, 89)])
def test_autograd_roots_against_eigenvalue_differences(gpu, kind, o, v, Q, seed):
    """torch.autograd through ADCEigen, against central differences (h = 1e-5)
    of the GPU's FP64 Davidson eigenvalues."""
    from paper_2511_21640_gb300.autograd import adc_roots
    x, nr = 0.4, 3
    p = _problem(o, v, Q, seed)
    B = torch.from_numpy(p.B.copy()).requires_grad_(True)
    eo = torch.from_numpy(p.eps_occ.copy()).requires_grad_(True)
    ev = torch.from_numpy(p.eps_vir.copy()).requires_grad_(True)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    wts = torch.tensor([1.0, -0.5, 0.25], dtype=torch.float64)
    om = adc_roots(B, eo, ev, xt, kind, 3, nr, 1e-10, "fp64", 1)
    (om * wts).sum().backward()
    rng = np.random.default_rng(5)
    dB = ograd.random_hermitian_direction(p.B.shape, 6)
    deo, dev = rng.standard_normal(o), rng.standard_normal(v)
    pred = ograd.directional(B.grad.numpy(), eo.grad.numpy(), ev.grad.numpy(), float(xt.grad), (dB, deo, dev, 0.7))
    h = 1e-5

    def roots(s):
        with gpu.Context(p.B + s * h * dB, p.eps_occ + s * h * deo, p.eps_vir + s * h * dev, kind=kind, order=3,
                         x=x + s * h * 0.7) as c:
            w, _, e64, _, rc = c.davidson(nr, tol=1e-10, precision="fp64", want_vectors=False)
            assert rc == 0
            return w

    fd = float(np.dot(wts.numpy(), (roots(1) - roots(-1)) / (2 * h)))
    assert abs(pred - fd) < 1e-6 * max(1.0, abs(fd)), (pred, fd)
