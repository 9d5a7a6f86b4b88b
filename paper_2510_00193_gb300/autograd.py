"""torch.autograd Functions over the C-ABI: the MTP energy as a
differentiable function of the positions and of the parameter vector theta
= [s | c | xi], with a hand-written backward (forces, dE/dtheta) and double
backward (directional second derivatives from the dual-number kernel), so
that a force-matching loss can be differentiated with respect to theta.

All arithmetic runs in the CUDA library; these classes only route tensors.
theta drives the potential: the forward pass and the double backward upload
it into the Potential handle (mtp_set_theta) before they evaluate, so a
training loop can update theta between steps without rebuilding the handle.
"""
from __future__ import annotations

import torch

from . import MTP_FP64, mtp_compute_efv, mtp_compute_efv_tangent, mtp_set_theta


class MTPEnergy(torch.autograd.Function):
    """E(x, theta); backward gives (dE/dx, dE/dtheta), itself differentiable once more."""

    @staticmethod
    def forward(ctx, x, theta, potential, nlist, z, cell, precision):
        mtp_set_theta(potential, theta.detach().contiguous())
        out = mtp_compute_efv(potential, nlist, x.detach(), z, cell, precision=precision, dtheta=True)
        ctx.save_for_backward(x, theta, out["forces"], out["dtheta"])
        ctx.info = (potential, nlist, z, cell, precision)
        return out["e_total"][0].clone()

    @staticmethod
    def backward(ctx, g_e):
        x, theta, forces, dtheta = ctx.saved_tensors
        gx, gth = MTPEnergyGrad.apply(x, theta, g_e, forces, dtheta, *ctx.info)
        return gx, gth, None, None, None, None, None


class MTPEnergyGrad(torch.autograd.Function):
    """(g dE/dx, g dE/dtheta) with dE/dx = -F; its backward uses the tangent
    kernel along the incoming gradient of dE/dx."""

    @staticmethod
    def forward(ctx, x, theta, g_e, forces, dtheta, potential, nlist, z, cell, precision):
        ctx.save_for_backward(x, theta, g_e, forces, dtheta)
        ctx.info = (potential, nlist, z, cell, precision)
        return -forces * g_e, dtheta * g_e

    @staticmethod
    def backward(ctx, g_gx, g_gth):
        x, theta, g_e, forces, dtheta = ctx.saved_tensors
        potential, nlist, z, cell, precision = ctx.info
        if g_gth is not None and bool(torch.any(g_gth != 0)):
            raise NotImplementedError("second derivatives along theta are not provided")
        if g_gx is None:
            return (None,) * 10
        mtp_set_theta(potential, theta.detach().contiguous())   # the parameters of this graph's forward
        tan = mtp_compute_efv_tangent(potential, nlist, x.detach(), z, cell, g_gx.contiguous(),
                                      precision=precision, force_tan=True)
        grad_x = -tan["force_tan"] * g_e          # g_e H v
        grad_theta = tan["dtheta_tan"] * g_e      # g_e d/dt dE/dtheta along v
        grad_ge = (-forces * g_gx).sum()
        return grad_x, grad_theta, grad_ge, None, None, None, None, None, None, None


def energy(potential, nlist, x, z, cell, theta, precision=MTP_FP64):
    """Differentiable total energy (0-d tensor) of one configuration."""
    return MTPEnergy.apply(x, theta, potential, nlist, z, cell, precision)
