"""Differentiable PDA: torch.autograd.Function around mcrt_solve_pda and mcrt_pda_adjoint.

T = PDA(log rho, kappa_R) for a disk whose Monte Carlo state (tallies, visit counts, hence the PDA
region and the boundary temperatures) is fixed; rho and kappa_R enter through D = 1/(3 rho kappa_R)
(Eq. 2). The backward pass is one adjoint solve with the (symmetric) PDA matrix and a face-wise
gradient kernel, both in the CUDA library. The adjoint uses the library's last PDA solve, so a disk
must not be solved again between a forward and its backward.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mcrt


class PDAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_rho, kappa_R, disk, opts):
        rho = torch.exp(log_rho.detach()).double().cpu().numpy()
        kr = kappa_R.detach().double().cpu().numpy()
        disk.solve_pda(rho=rho, kappa_R=kr, **(opts or {}))
        dev = log_rho.device
        if dev.type == "cuda":
            T = torch.empty(disk.nr, disk.ntheta, dtype=torch.float64, device=dev)
            torch.cuda.synchronize(dev)
            disk.temperatures_dev(T.data_ptr(), None, mcrt.T_PDA)
            torch.cuda.synchronize(dev)
        else:
            T = torch.from_numpy(disk.temperatures(mcrt.T_PDA)[0])
        ctx.disk = disk
        ctx.dev = dev
        return T.to(log_rho.dtype)

    @staticmethod
    def backward(ctx, grad_T):
        disk, dev = ctx.disk, ctx.dev
        if dev.type == "cuda":
            w = grad_T.detach().to(torch.float64).contiguous()
            gl = torch.empty_like(w)
            gk = torch.empty_like(w)
            torch.cuda.synchronize(dev)
            disk.pda_adjoint_dev(w.data_ptr(), gl.data_ptr(), gk.data_ptr())
            torch.cuda.synchronize(dev)
        else:
            g1, g2 = disk.pda_adjoint(grad_T.detach().double().numpy())
            gl, gk = torch.from_numpy(g1), torch.from_numpy(g2)
        return gl.to(grad_T.dtype), gk.to(grad_T.dtype), None, None


def pda_temperature(disk, log_rho, kappa_R, **opts):
    """Differentiable PDA temperatures of `disk` (see PDAFunction)."""
    return PDAFunction.apply(log_rho, kappa_R, disk, opts)
