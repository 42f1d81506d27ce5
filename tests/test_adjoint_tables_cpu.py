"""The term tables the device adjoint differentiates, evaluated on the CPU
with numpy and compared with the oracle: the amplitude numerators (csrc/ee.cu,
kT2N and kS2N) against the second-order doubles and singles, and the IP/EA
tables (csrc/adjoint.cu) against the oracle's main, coupling and satellite
blocks, together with the split of sum_r g_r y_r^H M y_r that the IP/EA adjoint
differentiates. Reads the C++ source as text; no GPU."""
import os
import re

import numpy as np
import pytest

from synthetic import make_problem
from oracle.integrals import Amplitudes, eri

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2511_21640_gb300", "csrc")
SRC = os.path.join(CSRC, "ee.cu")
OCC = set("ijklMNOPRSTW")


def _table(name, src=SRC):
    with open(src) as fh:
        text = fh.read()
    m = re.search(r"const Rows " + name + r" = \{(.*?)\};", text, re.S)
    assert m, name
    return re.findall(r'\{"([^"]+)",\s*"([^"]+)"\}', m.group(1))


def _coef(s):
    if "/" in s:
        p, q = s.split("/")
        return float(p) / float(q)
    return float(s)


def _eval(rows, B, o, amp, out):
    total = 0.0
    for c, prod in rows:
        facs = re.findall(r"(\w+)\(([^)]*)\)", prod)
        ops, labs = [], []
        for name, lab in facs:
            lab = lab.replace(",", "")
            if name == "v":
                ops.append(eri(B, o, "".join("o" if ch in OCC else "v" for ch in lab)))
            elif name == "t1":
                ops.append(amp.t1.transpose(2, 3, 0, 1))  # t1(ab,ij) = t_ij^ab
            else:
                raise AssertionError(name)
            labs.append(lab)
        total = total + _coef(c) * np.einsum(",".join(labs) + "->" + out, *ops)
    return total


@pytest.mark.parametrize("o,v,seed", [(3, 5, 1), (4, 6, 2)])
def test_amplitude_numerator_tables_match_oracle(o, v, seed):
    p = make_problem(o, v, 7, seed=seed, sigma=0.2)
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir, second_order=True)
    eo, ev = p.eps_occ, p.eps_vir
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    t2 = _eval(_table("kT2N"), p.B, o, amp, "ijab") / D2
    assert np.abs(t2 - amp.t2d).max() < 1e-13 * max(1.0, np.abs(amp.t2d).max())
    D1 = eo[:, None] - ev[None, :]
    s2 = _eval(_table("kS2N"), p.B, o, amp, "ia") / D1
    assert np.abs(s2 - amp.t2s).max() < 1e-13 * max(1.0, np.abs(amp.t2s).max())


def _tensor(amp, B, o, name, lab):
    if name == "v":
        return eri(B, o, "".join("o" if ch in OCC else "v" for ch in lab))
    if name in ("t1", "t1c", "t2", "t2c"):
        t = (amp.t1 if name[1] == "1" else amp.t2d).transpose(2, 3, 0, 1)  # t(ab,ij) = t_ij^ab
        return t.conj() if name.endswith("c") else t
    if name in ("s2", "s2c"):
        t = amp.t2s.T  # s2(a,i) = t2_i^a
        return t.conj() if name == "s2c" else t
    raise AssertionError(name)


def _eval_full(rows, amp, B, o, v, out):
    """Sum of coef * product with Kronecker deltas d(xy) as identity matrices."""
    total = 0.0
    for c, prod in rows:
        ops, labs = [], []
        for name, lab in re.findall(r"(\w+)\(([^)]*)\)", prod):
            lab = lab.replace(",", "")
            ops.append(np.eye(o if lab[0] in OCC else v) if name == "d" else _tensor(amp, B, o, name, lab))
            labs.append(lab)
        total = total + _coef(c) * np.einsum(",".join(labs) + "->" + out, *ops)
    return total


IPEA = os.path.join(CSRC, "adjoint.cu")


@pytest.mark.parametrize("kind,o,v,seed", [("EA", 3, 6, 5), ("IP", 4, 5, 6), ("EA", 4, 5, 7), ("IP", 3, 6, 8)])
def test_ipea_tables_match_oracle_blocks(kind, o, v, seed):
    from oracle import adc as oadc
    p = make_problem(o, v, 8, seed=seed, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))
    amp = Amplitudes(p.B, p.eps_occ, p.eps_vir)
    T = lambda name: _table("k%s_%s" % (kind, name), IPEA)  # noqa: E731
    L = "ab" if kind == "EA" else "ij"
    e1 = amp.ev if kind == "EA" else amp.eo
    W = (1.0 if kind == "EA" else -1.0) * 0.5 * (e1[:, None] - e1[None, :])
    ev = lambda name, out: _eval_full(T(name), amp, p.B, o, v, out)  # noqa: E731
    mb = oadc.main_block(kind, amp)
    scale = max(1.0, np.abs(mb[2]).max())
    assert np.abs(ev("M2", L) + W * ev("P2", L) - mb[2]).max() < 1e-13 * scale
    assert np.abs(ev("Y3", L) + W * ev("P3", L) - mb[3]).max() < 1e-13 * scale
    bl = oadc.Blocks(kind, p.B, p.eps_occ, p.eps_vir)
    if kind == "EA":
        iu, ju = np.triu_indices(v, 1)
        pk = lambda C: C[:, :, iu, ju].reshape(v, -1)  # noqa: E731
        S1 = ev("S1", "jabkcd")
        S1p = S1[:, iu, ju][:, :, :, iu, ju].reshape(o * iu.size, -1)
        lc = "ckde"
    else:
        iu, ju = np.triu_indices(o, 1)
        pk = lambda C: C[:, iu, ju, :].reshape(o, -1)  # noqa: E731
        S1 = ev("S1", "ijaklb")
        S1p = S1[iu, ju][:, :, iu, ju].reshape(iu.size * v, -1)
        lc = "kija"
    assert np.abs(pk(ev("C1", lc)) - bl.M12[1]).max() < 1e-13
    assert np.abs(pk(ev("C2", lc)) - bl.M12[2]).max() < 1e-13
    assert np.abs(S1p - bl.M22[1]).max() < 1e-13

    # sum_r g_r y^H M y = sum rho o M11 + Re sum Y1c C Y2 + sum g |y2|^2 d0 + x/4 sum Y2c S1 Y2
    x, k = 0.7, 3
    M = oadc.explicit_matrix(kind, 3, x, p.B, p.eps_occ, p.eps_vir, blocks=bl)
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((k, M.shape[0])) + 1j * rng.standard_normal((k, M.shape[0]))
    g = rng.standard_normal(k)
    ref = sum(g[r] * np.vdot(Y[r], M @ Y[r]) for r in range(k)).real
    n1 = bl.n1
    y1 = Y[:, :n1]
    rho = np.einsum("z,zp,zq->pq", g, y1.conj(), y1)
    Y2 = oadc.unpack2(kind, Y[:, n1:], o, v)
    Y1c, Y2c = g[:, None] * y1.conj(), g[:, None, None, None] * Y2.conj()
    C = ev("C1", lc) + x * ev("C2", lc)
    M11 = bl.M11[0] + bl.M11[2] + x * bl.M11[3]
    s1 = "zjab,jabkcd,zkcd->" if kind == "EA" else "zija,ijaklb,zklb->"
    parts = (np.sum(rho * M11).real + np.einsum("zc,c" + lc[1:] + ",z" + lc[1:] + "->", Y1c, C, Y2).real
             + np.sum(g[:, None] * np.abs(Y[:, n1:]) ** 2 * np.real(np.diag(bl.M22[0]))[None])
             + 0.25 * x * np.einsum(s1, Y2c, S1, Y2).real)
    assert abs(parts - ref) < 1e-12 * max(1.0, abs(ref))
