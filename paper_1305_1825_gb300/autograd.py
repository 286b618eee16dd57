"""torch.autograd.Function over the treecode energy.

``TreecodeEnergy.apply(q, xyz, params)`` builds the octree of the charges (all
mobile, no images: every charge is an independent leaf of the graph) on the
GPU, returns the total treecode energy E = (1/2) l_B sum_i q_i phi_i, and its
backward pass calls the hand-written adjoint kernel (bhmc_forces), which
returns dE/dq and dE/dxyz through the same traversal with the MAC decisions
held fixed.  Forces are -xyz.grad.
"""
from __future__ import annotations

import torch

from . import bhmc


class TreecodeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, xyz, params, precision=bhmc.PREC_F32):
        if q.dtype != torch.float64 or xyz.dtype != torch.float64 or not q.is_cuda or not xyz.is_cuda:
            raise TypeError("q and xyz must be float64 CUDA tensors")
        p = dict(params, image=None, shell=None)
        wl = dict(params=p, q=q.detach().contiguous(), xyz=xyz.detach().reshape(-1, 3).contiguous(),
                  n_mobile=q.numel(), n_fixed=0)
        c = bhmc.Context(wl, precision=precision, warps=8, layout=bhmc.LAYOUT_AOS)
        ctx.bh = c
        ctx.shape = xyz.shape
        return torch.tensor(c.energy(), dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx, grad_E):
        c = ctx.bh
        n = c.n_mobile
        dEdr = torch.empty((n, 3), dtype=torch.float64, device=grad_E.device)
        dEdq = torch.empty(n, dtype=torch.float64, device=grad_E.device)
        c.forces(dEdr, dEdq)
        torch.cuda.current_stream().synchronize()
        c.close()
        return grad_E * dEdq, (grad_E * dEdr).reshape(ctx.shape), None, None


def treecode_energy(q, xyz, params, precision=bhmc.PREC_F32):
    return TreecodeEnergy.apply(q, xyz, params, precision)
