"""The amplitude tables the device adjoint differentiates (csrc/ee.cu, kT2N
and kS2N) evaluated on the CPU with numpy and compared with the oracle's
second-order doubles and singles. Reads the C++ source as text; no GPU."""
import os
import re

import numpy as np
import pytest

from synthetic import make_problem
from oracle.integrals import Amplitudes, eri

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2511_21640_gb300", "csrc", "ee.cu")
OCC = set("ijklMNOPRSTW")


def _table(name):
    text = open(SRC).read()
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
