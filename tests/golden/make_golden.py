"""Writes tests/golden/oracle_eigenvalues.txt from the oracle alone.

The paper prints no worked example that synthetic inputs reproduce (its
tables are molecular results in real basis sets), so the stored values here
are the oracle's: the lowest eigenvalues of the explicit ADC matrices
(Sec. 2.1, Eqs. 7 and 10-12) and the MP2 energy (1/4 sum <ij||ab> t_ij^ab
with the first-order amplitudes of Sec. 2.4) of small seeded problems. The
test beside this file recomputes them, so that a later change to the
oracle's arithmetic shows up as a change to this file.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synthetic import make_problem  # noqa: E402
from oracle import adc, adc_ee  # noqa: E402
from oracle.integrals import Amplitudes  # noqa: E402

# (label, kind, nocc, nvir, naux, order, x, dd_order, seed, nroots)
CASES = [
    ("ip3", "IP", 3, 6, 9, 3, 1.0, 1, 101, 4),
    ("ip2x3", "IP", 4, 5, 8, 3, 0.5, 1, 102, 4),
    ("ea2", "EA", 3, 6, 9, 2, 0.0, 1, 103, 4),
    ("ea2x3", "EA", 2, 7, 10, 3, 0.5, 1, 104, 4),
    ("ee3", "EE", 2, 4, 7, 3, 1.0, 1, 105, 4),
    ("ee3_dd0", "EE", 2, 4, 7, 3, 1.0, 0, 106, 4),
    ("ee2x3", "EE", 3, 3, 6, 3, 0.4, 1, 107, 4),
]


def problem(case):
    _, kind, o, v, Q, order, x, dd, seed, nroots = case
    return make_problem(o, v, Q, seed=seed, sigma=0.15, occ_range=(-3.0, -0.3), vir_range=(0.1, 5.0))


def values(case):
    _, kind, o, v, Q, order, x, dd, seed, nroots = case
    p = problem(case)
    if kind == "EE":
        M = adc_ee.explicit_matrix(order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd)
    else:
        M = adc.explicit_matrix(kind, order, x, p.B, p.eps_occ, p.eps_vir)
    w = np.linalg.eigvalsh(M)[:nroots]
    e2 = Amplitudes(p.B, p.eps_occ, p.eps_vir).mp2_energy()
    return float(np.real(e2)), [float(a) for a in w]


def main():
    lines = ["# lowest eigenvalues of the explicit ADC matrices and MP2 energies (Eh), written by",
             "# tests/golden/make_golden.py from the oracle (Sec. 2.1 Eqs. 7, 10-12; E2 = 1/4 sum <ij||ab> t_ij^ab",
             "# with the first-order amplitudes of Sec. 2.4, Eq. 25)",
             "# label kind nocc nvir naux order x dd_order seed | E2 | omega_1 .. omega_n"]
    for case in CASES:
        e2, w = values(case)
        head = " ".join(str(c) for c in case[:9])
        lines.append(f"{head} | {e2:.15e} | " + " ".join(f"{a:.15e}" for a in w))
    with open(os.path.join(HERE, "oracle_eigenvalues.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
