"""Differentiable far-field objective of the ET-AIM march (torch.autograd).

J(a) = sum_n sum_d sum_q |F_q(n; r_d)|^2, where the march of Eq. 5 is driven by the
incident envelope samples a (complex128 [n_samp]) and F is the far-field envelope of
the marched currents.  Both passes are single library calls and neither stores a
history of N_t steps:

* forward, aim_march_farfield: the march adds each committed step's contribution to F
  at once, so only F and the march's own N_g-step history exist;
* backward, aim_march_adjoint_farfield: the adjoint march M^H lam = A^H F runs in
  reversed time (the transposed march of the conjugated source, conjugated), forming
  each step's source from F and adding each lam_l into the gradient B^H lam at once.

This module only orders the calls.  PyTorch's convention for a real loss of complex
inputs: a.grad = 2 dJ/d conj(a) (so that dJ = Re(sum conj(a.grad) da)).
"""
from __future__ import annotations

import torch

from . import abi


class FarFieldObjective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a, handle, wave, dirs, n_steps, tol, i0, n0, n_out):
        khat, phat = wave
        rhat, e1, e2 = dirs
        F, _, _ = abi.aim_march_farfield(handle, khat, phat, i0, a.detach().contiguous(), n_steps, tol,
                                         rhat, e1, e2, n0, n_out)
        fctx.save_for_backward(F)
        fctx.meta = (handle, wave, dirs, n_steps, tol, i0, n0, a.shape[0])
        return (F.abs() ** 2).sum()

    @staticmethod
    def backward(fctx, gJ):
        (F,) = fctx.saved_tensors
        handle, (khat, phat), (rhat, e1, e2), n_steps, tol, i0, n0, n_samp = fctx.meta
        g, _, _ = abi.aim_march_adjoint_farfield(handle, khat, phat, i0, n_samp, n_steps, tol, rhat, e1, e2, n0,
                                                 F.contiguous())
        return 2.0 * gJ * g, None, None, None, None, None, None, None, None


def far_field_objective(a, ctx, wave, dirs, n_steps, tol, i0, n0, n_out):
    """J(a) with autograd support.  ctx: AimContext; wave = (khat, phat); dirs =
    (rhat, e1, e2) as [nd, 3] arrays; samples a_i for i = i0..i0+len(a)-1; F over
    n = n0..n0+n_out-1."""
    return FarFieldObjective.apply(a, ctx.handle, wave, dirs, n_steps, tol, i0, n0, n_out)
