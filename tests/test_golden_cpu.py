"""The oracle reproduces the stored values of tests/golden/oracle_eigenvalues.txt
(written by tests/golden/make_golden.py from the oracle): lowest eigenvalues
of the explicit IP, EA and EE matrices at ADC(2), ADC(2)+x(3) and ADC(3)
(Sec. 2.1, Eqs. 7, 10-12) and the MP2 energy, to 1e-12 Eh. A change to the
oracle's arithmetic shows up here and has to be made on purpose, with the
file rewritten by the script."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def _stored():
    rows = {}
    with open(os.path.join(HERE, "golden", "oracle_eigenvalues.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            head, e2, w = ln.split("|")
            rows[head.split()[0]] = (float(e2), [float(a) for a in w.split()])
    return rows


@pytest.mark.parametrize("case", make_golden.CASES, ids=[c[0] for c in make_golden.CASES])
def test_oracle_reproduces_golden(case):
    e2_ref, w_ref = _stored()[case[0]]
    e2, w = make_golden.values(case)
    assert abs(e2 - e2_ref) < 1e-12
    assert np.abs(np.array(w) - np.array(w_ref)).max() < 1e-12
