"""Differentiable susceptibility: chi(k) at the end of a flow as a torch.autograd.Function of
linear coupling parameters theta (couplings M_c = sum_p theta_p B[p, c]).

The forward pass integrates the tangent-linear flow on the GPU (sr_flow_init_tangent: every
kernel propagates d/dtheta_p exactly with dual numbers) and stores the Jacobian
d chi(k) / d theta; the backward pass contracts it with the incoming gradient.  With two
parameters the forward-mode Jacobian costs one flow of dual numbers and needs no stored
trajectory (no checkpoints).
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import SR_EULER, SR_FP64, SR_SU2, SR_XYZ, Flow, Lattice


class SusceptibilityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, cell, sites, B, L, mesh, lambdas, kpts, backend):
        th = theta.detach().cpu().double().numpy()
        M = np.einsum("p,pcij->cij", th, B)
        coups = [(f, t, M[c]) for c, (f, t) in enumerate(sites)]
        lat = Lattice(cell.prim, cell.basis, cell.bonds, coups, L, backend)
        fl = Flow(lat, mesh, float(lambdas[0]), SR_FP64, tangents=B)
        for lam in lambdas[1:]:
            fl.step(float(lam), SR_EULER)
        chi, dchi = fl.measure_tangent(kpts)
        fl.close()
        ctx.save_for_backward(torch.as_tensor(dchi, dtype=theta.dtype))
        return torch.as_tensor(chi, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (dchi,) = ctx.saved_tensors
        return (grad_out @ dchi.to(grad_out.device), None, None, None, None, None, None, None, None)


def susceptibility(theta: torch.Tensor, cell, sites, B, L: int, mesh, lambdas, kpts, backend: int = SR_XYZ):
    """chi(k) (tensor of len(kpts)) differentiable in theta."""
    return SusceptibilityFn.apply(theta, cell, sites, np.asarray(B, dtype=np.float64), L,
                                  np.asarray(mesh, dtype=np.float64), np.asarray(lambdas, dtype=np.float64),
                                  np.asarray(kpts, dtype=np.float64), backend)
