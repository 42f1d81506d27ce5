"""Eigenvalue derivatives of the ADC matrix (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For a non-degenerate root omega_r of the Hermitian matrix M(theta) with
normalised eigenvector y_r (Eq. 10), the Hellmann-Feynman theorem gives

    d omega_r / d theta = y_r^H (dM/dtheta) y_r.

The inputs theta are the Cholesky vectors B (complex, Hermitian in p, q for
every Q), the orbital energies and x. Along a direction (dB, deo, dev, dx)
the derivative of the matrix is taken here by central differences of the
explicit matrix, M(theta + h D) - M(theta - h D) over 2h, whose error is
O(h^2) (every matrix element is a smooth function of the inputs), and
contracted with the eigenvectors of M(theta). M is linear in x, so the x
component of the difference is exact.

A gradient g_B of a real function in the convention of complex automatic
differentiation (the derivative with respect to the real part plus i times
the derivative with respect to the imaginary part, for every element)
predicts the directional derivative sum Re(conj(g_B) dB) + g_eo . deo +
g_ev . dev + g_x dx; ``directional`` is that value for given gradients.
"""
from __future__ import annotations

import numpy as np

from synthetic import random_hermitian_direction  # noqa: F401  (seeded input generator, re-exported)

from . import adc as _adc
from . import adc_ee as _ee

__all__ = ["matrix", "hf_directional", "eig_fd_directional", "directional", "random_hermitian_direction"]


def matrix(kind, order, x, B, eps_occ, eps_vir, dd_order=1):
    """Explicit ADC matrix of any kind (small cases only)."""
    if kind == "EE":
        return _ee.explicit_matrix(order, x, B, eps_occ, eps_vir, dd_order=dd_order)
    return _adc.explicit_matrix(kind, order, x, B, eps_occ, eps_vir)


def _shift(B, eo, ev, x, D, s):
    dB, deo, dev, dx = D
    return (B + s * dB if dB is not None else B, eo + s * deo if deo is not None else eo,
            ev + s * dev if dev is not None else ev, x + s * dx)


def hf_directional(kind, order, x, B, eps_occ, eps_vir, nroots, D, h=1e-5, dd_order=1, Y=None):
    """y_r^H [M(theta + hD) - M(theta - hD)] / 2h y_r for the lowest nroots roots.

    D = (dB, deo, dev, dx), each None/0 for no change. Y: eigenvectors to use
    ([nroots][N]); by default the eigenvectors of M(theta). Returns (dw, w, Y)."""
    M0 = matrix(kind, order, x, B, eps_occ, eps_vir, dd_order)
    w, V = np.linalg.eigh(M0)
    if Y is None:
        Y = V[:, :nroots].T
    Mp = matrix(kind, order, *_reorder(_shift(B, eps_occ, eps_vir, x, D, +h)), dd_order=dd_order)
    Mm = matrix(kind, order, *_reorder(_shift(B, eps_occ, eps_vir, x, D, -h)), dd_order=dd_order)
    dM = (Mp - Mm) / (2 * h)
    dw = np.real(np.einsum("rp,pq,rq->r", Y.conj(), dM, Y))
    return dw, w[:nroots], Y


def _reorder(t):
    B, eo, ev, x = t
    return x, B, eo, ev


def eig_fd_directional(kind, order, x, B, eps_occ, eps_vir, nroots, D, h=1e-4, dd_order=1):
    """Central difference of the lowest nroots eigenvalues along D."""
    wp = np.linalg.eigvalsh(matrix(kind, order, *_reorder(_shift(B, eps_occ, eps_vir, x, D, +h)),
                                   dd_order=dd_order))[:nroots]
    wm = np.linalg.eigvalsh(matrix(kind, order, *_reorder(_shift(B, eps_occ, eps_vir, x, D, -h)),
                                   dd_order=dd_order))[:nroots]
    return (wp - wm) / (2 * h)


def directional(gB, geo, gev, gx, D):
    """The directional derivative that gradients (gB, geo, gev, gx) predict along D."""
    dB, deo, dev, dx = D
    s = 0.0
    if dB is not None:
        s += float(np.real(np.vdot(gB, dB)))
    if deo is not None:
        s += float(np.dot(geo, deo))
    if dev is not None:
        s += float(np.dot(gev, dev))
    return s + float(gx) * float(dx)
