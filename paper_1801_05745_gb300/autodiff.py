"""torch.autograd support: kappa map and its variance and skewness as
differentiable functions of theta = (Omega_m, h, alpha, beta, z0), with the
particle counts held fixed.  The backward pass is the library's adjoint
(ufc_kappa_backward); the forward pass is ufc_kappa_coeffs + ufc_kappa_stats.

The gradient is that of the unrounded map kappa_p = sum_b A_b n_bp - C; the
forward's variance and skewness are moments of the FP32 map (they differ by
FP32 rounding only).
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class KappaStats(torch.autograd.Function):
    """(kappa [npix] FP32, var, skew) = f(theta) for fixed counts."""

    @staticmethod
    def forward(ctx_, theta, counts, lib, boxes, z_edges, nside, source_kind, z_s, z_max,
                units_mpc_over_h, pdf_range):
        t = theta.detach().cpu().double().numpy()
        cosmo = api.make_cosmo(t[0], t[1], units_mpc_over_h)
        src = api.make_source(kind=source_kind, z_s=z_s, alpha=t[2], beta=t[3], z0=t[4],
                              z_max=z_max)
        A, B, C, dA, dC = api.kappa_coeffs(cosmo, boxes, z_edges, nside, src, derivs=True)
        lo, hi = pdf_range
        kap, mom, _ = lib.kappa_stats(counts, A, C, lo, hi, 16)
        m = mom.cpu().numpy()
        ctx_.lib, ctx_.counts = lib, counts
        ctx_.coef = (A, C, dA, dC)
        ctx_.theta_dtype = theta.dtype
        var = torch.tensor(m[1], dtype=torch.float64)
        skew = torch.tensor(m[4], dtype=torch.float64)
        return kap, var, skew

    @staticmethod
    def backward(ctx_, g_kappa, g_var, g_skew):
        A, C, dA, dC = ctx_.coef
        gk = None
        if g_kappa is not None and bool(torch.any(g_kappa != 0)):
            gk = g_kappa.detach().float().contiguous()
        wv = float(g_var) if g_var is not None else 0.0
        ws = float(g_skew) if g_skew is not None else 0.0
        grad, _, _ = ctx_.lib.kappa_backward(ctx_.counts, A, C, dA, dC, wv, ws, gk)
        gt = torch.from_numpy(np.asarray(grad)).to(ctx_.theta_dtype)
        return (gt,) + (None,) * 10


def kappa_stats(theta, counts, lib, boxes, z_edges, nside, source_kind=1, z_s=1.5, z_max=1.5,
                units_mpc_over_h=1, pdf_range=(-1.0, 1.0)):
    """Differentiable (kappa, var, skew); theta = tensor([Om, h, alpha, beta, z0])."""
    return KappaStats.apply(theta, counts, lib, boxes, z_edges, nside, source_kind, z_s, z_max,
                            units_mpc_over_h, pdf_range)
