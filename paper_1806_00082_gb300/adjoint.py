"""The differentiation form as a torch.autograd.Function.

theta [n_pot, 3 nb + ns] (tanh-edged barriers and segment offsets, see
include/wmc.h) -> potential V -> kernel rows VWh [n_pot n_x, Q/2] and gamma
[n_pot n_x].  Forward and backward run in libwmc (wmc_potential_tanh,
wmc_kernel_eval_rows, wmc_kernel_cdf; wmc_kernel_vjp, wmc_potential_tanh_vjp).
"""
from __future__ import annotations

import torch

from . import wmc


class KernelOfPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, p, n_barriers, n_segments, eps_nm, ws):
        theta = theta.detach().contiguous().float()
        V = wmc.potential_tanh(p, theta, n_barriers, n_segments, eps_nm)
        VWh = wmc.kernel_eval_rows(p, V, ws)
        _, gamma, _ = wmc.kernel_cdf(p, VWh, with_cdf=False)
        ctx.save_for_backward(theta, VWh)
        ctx.cfg = (p, n_barriers, n_segments, eps_nm, ws)
        return VWh, gamma.float()

    @staticmethod
    def backward(ctx, gVW, g_gamma):
        theta, VWh = ctx.saved_tensors
        p, nb, ns, eps, ws = ctx.cfg
        gv = gVW.contiguous().float() if gVW is not None else None
        gg = g_gamma.contiguous().float() if g_gamma is not None else None
        if gv is None and gg is None:
            return None, None, None, None, None, None
        Vbar = wmc.kernel_vjp(p, VWh, gv, gg, theta.shape[0], ws)
        tb = wmc.potential_tanh_vjp(p, theta, nb, ns, eps, Vbar)
        return tb, None, None, None, None, None


def kernel_of_potential(theta: torch.Tensor, p: wmc.Params, n_barriers: int, n_segments: int, eps_nm: float,
                        ws: torch.Tensor):
    """(VWh, gamma) of the potentials described by theta, differentiable in theta."""
    return KernelOfPotential.apply(theta, p, n_barriers, n_segments, eps_nm, ws)
