"""torch.autograd binding of the discrete adjoint: the absorbed energy in a target region as a
differentiable function of per-block absorption and scattering coefficients.

Forward and backward both run the library (kitrt_adjoint computes J and its gradient in one
forward-and-reverse sweep with checkpoints); autograd only routes the gradient.
"""
from __future__ import annotations

import torch


class AbsorbedEnergy(torch.autograd.Function):
    """J(sigma_a_blk, sigma_s_blk) for a fixed solver, mesh partition, source and target."""

    @staticmethod
    def forward(ctx, sigma_a_blk, sigma_s_blk, solver, u0, alpha0, q, block_of_cell, target, dt,
                nsteps, ckpt_every):
        sa = sigma_a_blk.detach()[block_of_cell.long()].contiguous()
        ss = sigma_s_blk.detach()[block_of_cell.long()].contiguous()
        J, gsa, gss = solver.adjoint(u0, alpha0, sa, ss, q, block_of_cell, sigma_a_blk.numel(), target,
                                     dt, nsteps, ckpt_every)
        dev = sigma_a_blk.device
        ctx.save_for_backward(torch.from_numpy(gsa).to(dev), torch.from_numpy(gss).to(dev))
        return torch.tensor(J, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        gsa, gss = ctx.saved_tensors
        return gJ * gsa, gJ * gss, None, None, None, None, None, None, None, None, None


def absorbed_energy(sigma_a_blk, sigma_s_blk, solver, u0, alpha0, q, block_of_cell, target, dt,
                    nsteps, ckpt_every=16):
    return AbsorbedEnergy.apply(sigma_a_blk, sigma_s_blk, solver, u0, alpha0, q, block_of_cell,
                                target, dt, nsteps, ckpt_every)
