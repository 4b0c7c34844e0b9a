"""Differentiable far-field objective of the ET-AIM march (torch.autograd).

J(a) = sum_n sum_d sum_q |F_q(n; r_d)|^2, where the march of Eq. 5 is driven by the
incident envelope samples a (complex128 [n_samp]) and F is the far-field envelope of
the marched currents.  The forward pass runs the march on the device and keeps only
F (the march itself holds just its N_g-step history); the backward pass runs the
adjoint march M^H lam = dJ/d conj(I) -- the transposed march of the conjugated
source in reversed time -- and maps lam back to the samples.  All steps run in the
CUDA library; this module only orders the calls.

PyTorch's convention for a real loss of complex inputs: a.grad = 2 dJ/d conj(a)
(so that dJ = Re(sum conj(a.grad) da)).
"""
from __future__ import annotations

import torch

from . import abi


class FarFieldObjective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a, handle, wave, dirs, n_steps, tol, i0, n0, n_out):
        khat, phat = wave
        rhat, e1, e2 = dirs
        a_ = a.detach().contiguous()
        V = abi.aim_excitation_samples(handle, khat, phat, i0, a_, n_steps)
        I, _, _ = abi.aim_march_source(handle, V.reshape(n_steps, 1, -1), tol)
        F = abi.aim_farfield(handle, rhat, e1, e2, I.reshape(n_steps, -1), n0, n_out)
        fctx.save_for_backward(F)
        fctx.meta = (handle, wave, dirs, n_steps, tol, i0, n0, a.shape[0])
        return (F.abs() ** 2).sum()

    @staticmethod
    def backward(fctx, gJ):
        (F,) = fctx.saved_tensors
        handle, (khat, phat), (rhat, e1, e2), n_steps, tol, i0, n0, n_samp = fctx.meta
        G = abi.aim_farfield_adjoint(handle, rhat, e1, e2, n_steps, n0, F)          # dJ/d conj(I)
        src = torch.flip(G, dims=[0]).conj().resolve_conj().contiguous().reshape(n_steps, 1, -1)
        u, _, _ = abi.aim_march_source(handle, src, tol, transpose=True)
        lam = torch.flip(u, dims=[0]).conj().resolve_conj().contiguous().reshape(n_steps, -1)  # M^H lam = G
        g = abi.aim_excitation_samples_adjoint(handle, khat, phat, i0, n_samp, lam)
        return 2.0 * gJ * g, None, None, None, None, None, None, None, None


def far_field_objective(a, ctx, wave, dirs, n_steps, tol, i0, n0, n_out):
    """J(a) with autograd support.  ctx: AimContext; wave = (khat, phat); dirs =
    (rhat, e1, e2) as [nd, 3] arrays; samples a_i for i = i0..i0+len(a)-1; F over
    n = n0..n0+n_out-1."""
    return FarFieldObjective.apply(a, ctx.handle, wave, dirs, n_steps, tol, i0, n0, n_out)
