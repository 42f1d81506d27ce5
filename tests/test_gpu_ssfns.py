"""State-specific natural spinors on the GPU (Sec. 2.4, Eqs. 31-32) against the
oracle (oracle/ssfns.py): the state density (1e-12), the natural spinors of
D^MP2 + D^state (as the MP2 ones: occupations 1e-12, semicanonical energies
1e-10, kept projector 1e-9), the carried-over guess for a given U (1e-12),
the root-specific Davidson (1e-8 Eh against the explicit matrix's eigenpair of
largest overlap) and the whole procedure (every energy of Eq. 32 to 1e-8 Eh,
the same number of kept spinors).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_problem  # noqa: E402
from oracle import ssfns as oss  # noqa: E402
from oracle.fns import fns_basis, fns_density  # noqa: E402


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_2511_21640_gb300 as m
    return m


def _problem(o, v, Q, seed):
    return make_problem(o, v, Q, seed=seed, sigma=0.12, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))


def _unit(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return y / np.linalg.norm(y)


@pytest.mark.parametrize("kind,o,v,Q,seed", [("EA", 3, 6, 10, 61), ("EE", 3, 5, 9, 62), ("EA", 1, 4, 6, 63)])
def test_state_density_and_ssfns_basis(gpu, kind, o, v, Q, seed):
    p = _problem(o, v, Q, seed)
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=2) as c:
        y = _unit(c.N, seed + 1)
        D = c.state_density(y)
        Dref = oss.state_density(kind, y, o, v)
        assert np.abs(D - Dref).max() < 1e-12
        Dss = fns_density(p.B, p.eps_occ, p.eps_vir) + Dref
        eta_r, _, _, _, _ = fns_basis(Dss, p.eps_vir, -1.0)
        crit = float(np.sqrt(eta_r[v - 2] * eta_r[v - 3]))  # keep v - 2
        eta_r, _, nk_r, U_r, e_r = fns_basis(Dss, p.eps_vir, crit)
        r = c.ssfns_density(y, crit)
        assert np.abs(r["D"] - Dss).max() < 1e-12 * max(1.0, np.abs(Dss).max())
        assert np.abs(r["eta"] - eta_r).max() < 1e-12 * max(1.0, eta_r.max())
        assert r["n_keep"] == nk_r == v - 2
        assert np.abs(r["eps_new"] - e_r).max() < 1e-10
        assert np.abs(r["U"] @ r["U"].conj().T - U_r @ U_r.conj().T).max() < 1e-9
        g = c.fns_vector(y, r["U"])
        gref = oss.to_fns_basis(kind, y, o, v, r["U"])
        assert np.abs(g - gref).max() < 1e-12


@pytest.mark.parametrize("kind,o,v,Q,target,seed", [("EA", 4, 10, 16, 2, 64), ("EE", 3, 6, 10, 3, 65)])
def test_davidson_follow(gpu, kind, o, v, Q, target, seed):
    p = _problem(o, v, Q, seed)
    M = oss.matrix(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir)
    w, V = np.linalg.eigh(M)
    g = V[:, target] + 0.3 * V[:, target + 1] + 0.05 * _unit(M.shape[0], seed)
    g = g / np.linalg.norm(g)
    wr, xr, r, ov = oss.follow_root(M, g)
    assert r == target
    with gpu.Context(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=0.5) as c:
        om, y, e64, st, rc = c.davidson_follow(g, tol=1e-9, max_iter=400)
    assert rc == 0 and e64 <= 1e-9
    assert abs(om - wr) < 1e-8
    assert abs(abs(np.vdot(xr, y)) - 1.0) < 1e-8


def _crit_away_from(etas):
    """A threshold in a wide gap of every root's occupation spectrum (mid-range)."""
    best, bc = -1.0, None
    e0 = np.sort(etas[0])[::-1]
    n = e0.size
    for i in range(n // 3, n - 1):
        c = float(np.sqrt(e0[i] * e0[i + 1]))
        if not c > 0:
            continue
        d = min(np.abs(np.log(np.maximum(e, 1e-300)) - np.log(c)).min() for e in etas)
        if d > best:
            best, bc = d, c
    return bc


@pytest.mark.parametrize("kind,o,v,Q,seed", [("EA", 3, 8, 12, 66), ("EE", 2, 6, 10, 67)])
def test_ssfns_procedure(gpu, kind, o, v, Q, seed):
    p = _problem(o, v, Q, seed)
    nroots = 2
    etas = [r["eta"] for r in oss.ssfns(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir, nroots, eta_crit=-1.0)]
    crit = _crit_away_from(etas)
    ref = oss.ssfns(kind, 3, 0.5, p.B, p.eps_occ, p.eps_vir, nroots, eta_crit=crit)
    out = gpu.ssfns(p.B, p.eps_occ, p.eps_vir, kind=kind, order=3, x=0.5, nroots=nroots, eta_crit=crit, tol=1e-10,
                    max_iter=400)
    assert any(q["n_keep"] < v for q in ref)  # at least one root really truncated
    for r, q in zip(out, ref):
        assert r["status"] == 0
        assert r["n_keep"] == q["n_keep"] and 0 < r["n_keep"] <= v
        for key in ("omega2_canonical", "omega2_fns", "omega_fns", "omega_corrected"):
            assert abs(r[key] - q[key]) < 1e-8, (key, r[key], q[key])
