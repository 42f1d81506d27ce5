"""Roots of the ADC matrix as a differentiable torch function.

``ADCEigen.apply(B, eps_occ, eps_vir, x, kind, order, nroots, tol, precision,
dd_order)`` returns the lowest ``nroots`` roots (a float64 tensor). The
forward pass is one ``adc_init`` + ``adc_davidson`` (with eigenvectors); the
backward pass is ``adc_sigma_adjoint`` (Hellmann-Feynman, Eq. 10), giving the
gradients with respect to B (complex, torch's convention), the orbital
energies and x. Valid for non-degenerate roots. All arithmetic runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context


class ADCEigen(torch.autograd.Function):
    @staticmethod
    def forward(ctx, B, eps_occ, eps_vir, x, kind="EE", order=3, nroots=4, tol=1e-8, precision="fp64",
                dd_order=1):
        dev = B.device
        Bh = B.detach().cpu().numpy()
        eo = eps_occ.detach().cpu().numpy().astype(np.float64)
        ev = eps_vir.detach().cpu().numpy().astype(np.float64)
        xv = float(x.detach().cpu()) if torch.is_tensor(x) else float(x)
        c = Context(Bh, eo, ev, kind=kind, order=order, x=xv, dd_order=dd_order)
        om, Y, e64, st, rc = c.davidson(nroots, tol=tol, precision=precision, want_vectors=True)
        ctx.c, ctx.Y, ctx.dev = c, Y, dev
        ctx.x_is_tensor = torch.is_tensor(x)
        return torch.from_numpy(om.copy()).to(dev)

    @staticmethod
    def backward(ctx, gomega):
        g = gomega.detach().cpu().numpy().astype(np.float64)
        gB, geo, gev, gx = ctx.c.sigma_adjoint(ctx.Y, g)
        ctx.c.close()
        dev = ctx.dev
        gxt = torch.tensor(gx, dtype=torch.float64, device=dev) if ctx.x_is_tensor else None
        return (torch.from_numpy(gB).to(dev), torch.from_numpy(geo).to(dev), torch.from_numpy(gev).to(dev), gxt,
                None, None, None, None, None, None)


def adc_roots(B, eps_occ, eps_vir, x, kind="EE", order=3, nroots=4, tol=1e-8, precision="fp64", dd_order=1):
    """Differentiable lowest roots (see ADCEigen)."""
    return ADCEigen.apply(B, eps_occ, eps_vir, x, kind, order, nroots, tol, precision, dd_order)
