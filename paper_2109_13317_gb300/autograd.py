"""Differentiable susceptibility: chi(k) at the end of a flow as a torch.autograd.Function of
linear coupling parameters theta (couplings M_c = sum_p theta_p B[p, c]).

Two ways to the same derivative:

* ``susceptibility_adjoint`` (reverse mode): the forward pass integrates the FP64 flow with
  Euler steps and keeps the state every ``every`` steps; the backward pass starts from
  d chi / d state at the final cutoff (sr_measure_susceptibility_adjoint), walks the steps
  backwards (sr_flow_step_adjoint), recomputing the states of one checkpoint segment at a
  time, and contracts the adjoint of the initial vertex with d Gamma_init / d theta
  (sr_flow_initial_vertex_adjoint: the initial vertex is J / 4, linear in the couplings).
  The couplings themselves come from theta through sr_couplings_linear.  Memory: one state per checkpoint plus
  one segment; cost: one extra forward flow plus the adjoint steps, independent of the
  number of parameters.
* ``susceptibility`` (forward mode): the tangent-linear flow (sr_flow_init_tangent: every
  kernel propagates d/dtheta_p with dual numbers) gives the Jacobian d chi(k) / d theta in the
  forward pass; cheap for the two parameters of a coupling sweep, no stored trajectory.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import SR_EULER, SR_FP64, SR_SU2, SR_XYZ, Flow, Lattice, sr_couplings_linear


class SusceptibilityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, cell, sites, B, L, mesh, lambdas, kpts, backend):
        M = sr_couplings_linear(theta.detach().cpu().double().numpy(), B)
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


class SusceptibilityAdjointFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, cell, sites, B, L, mesh, lambdas, kpts, backend, every):
        M = sr_couplings_linear(theta.detach().cpu().double().numpy(), B)
        coups = [(f, t, M[c]) for c, (f, t) in enumerate(sites)]
        lat = Lattice(cell.prim, cell.basis, cell.bonds, coups, L, backend)
        fl = Flow(lat, mesh, float(lambdas[0]), SR_FP64)
        ckpt = {0: tuple(x.clone() for x in fl.get_state())}
        nstep = len(lambdas) - 1
        for n in range(1, nstep + 1):
            fl.step(float(lambdas[n]), SR_EULER)
            if n % every == 0 and n < nstep:
                ckpt[n] = tuple(x.clone() for x in fl.get_state())
        chi, _ = fl.measure(kpts, want_ij=False)
        final = tuple(x.clone() for x in fl.get_state())
        ctx.state = (lat, fl, ckpt, final, B, mesh, lambdas, kpts, every)
        return torch.as_tensor(chi, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        lat, fl, ckpt, final, B, mesh, lambdas, kpts, every = ctx.state
        nstep = len(lambdas) - 1
        fl.set_state(float(lambdas[-1]), *final)
        bar_s, bar_G = fl.measure_adjoint(kpts, grad_out.detach().cpu().double().numpy())
        for start in sorted(ckpt, reverse=True):
            end = min(start + every, nstep)
            states = [ckpt[start]]
            fl.set_state(float(lambdas[start]), *ckpt[start])
            for n in range(start + 1, end):
                fl.step(float(lambdas[n]), SR_EULER)
                states.append(tuple(x.clone() for x in fl.get_state()))
            for n in range(end - 1, start - 1, -1):
                fl.set_state(float(lambdas[n]), *states[n - start])
                fl.step_adjoint(float(lambdas[n]), float(lambdas[n + 1]), bar_s, bar_G)
        # the initial vertex J / 4 is linear in theta: contract its derivative with bar_G
        grad = torch.as_tensor(fl.initial_vertex_adjoint(B, bar_G), dtype=grad_out.dtype)
        return (grad, None, None, None, None, None, None, None, None, None)


def susceptibility_adjoint(theta: torch.Tensor, cell, sites, B, L: int, mesh, lambdas, kpts,
                           backend: int = SR_XYZ, every: int = 20):
    """chi(k) (tensor of len(kpts)) differentiable in theta by the reverse-mode adjoint flow
    with a checkpoint every `every` Euler steps."""
    if every < 1:
        raise ValueError("every must be >= 1")
    return SusceptibilityAdjointFn.apply(theta, cell, sites, np.asarray(B, dtype=np.float64), L,
                                         np.asarray(mesh, dtype=np.float64), np.asarray(lambdas, dtype=np.float64),
                                         np.asarray(kpts, dtype=np.float64), backend, int(every))
