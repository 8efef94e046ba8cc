"""Differentiable dose + cost (Eq. 1-3) as torch.autograd.Functions.

Forward and backward run in libvmat's kernels; this module only passes
tensors.  Batches hold 32 vectors, laid out row-major as the kernels want:
fluence X [B, 32] (column b = fluence vector b), intensities Y [N, 32].

  dose_cost(plan, X)              cost_b = sum_j F((D^T X)_jb)            (Eq. 1)
      d cost_b / d X[:, b] = D F'(z_b)                  (the beamlet prices)
  aperture_dose_cost(plan, Y, l, r)
      cost_b = sum_j F((D^T A Y)_jb) + gamma G(Y[:, b])                    (Eq. 3)
      d cost_b / d Y[:, b] = A^T D F'(z_b) + gamma dG(Y[:, b])
A is the aperture map of the leaves l, r [N*R] (int16, on the device).
"""
from __future__ import annotations

import torch

from . import vmat


class _DoseCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, plan):
        Z, Fp, cost = plan.dose_batch32(X.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(Fp)
        return torch.as_tensor(cost, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, gcost):
        (Fp,) = ctx.saved_tensors
        w = gcost.to(torch.float32).contiguous()
        G = ctx.plan.price_batch32(Fp, w)
        return G.view(ctx.plan.cfg.n_beamlets, 32), None


class _ApertureDoseCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, plan, l, r):
        Y = Y.contiguous()
        X = torch.empty(plan.cfg.n_beamlets, 32, dtype=torch.float32, device=Y.device)
        Z = torch.empty(plan.prob.n_vox, 32, dtype=torch.float32, device=Y.device)
        Fp = torch.empty_like(Z)
        cost = vmat.vmat_aperture_dose_cost_batch32(plan.ctx, l, r, Y, X, Z, Fp)
        ctx.plan = plan
        ctx.save_for_backward(Fp, Y, l, r)
        return torch.as_tensor(cost, dtype=torch.float64, device=Y.device)

    @staticmethod
    def backward(ctx, gcost):
        Fp, Y, l, r = ctx.saved_tensors
        plan = ctx.plan
        w = gcost.to(torch.float32).contiguous()
        GX = plan.price_batch32(Fp, w)
        GY = torch.empty(plan.cfg.n_angles, 32, dtype=torch.float32, device=Y.device)
        vmat.vmat_aperture_adjoint_batch32(plan.ctx, l, r, GX, GY, Y, w)
        return GY, None, None, None


def dose_cost(plan, X):
    """cost [32] (float64) of 32 fluence vectors X [B, 32] (float32, CUDA)."""
    if X.shape != (plan.cfg.n_beamlets, 32) or X.dtype != torch.float32 or not X.is_cuda:
        raise ValueError("X must be a CUDA float32 tensor of shape [B, 32]")
    return _DoseCost.apply(X, plan)


def aperture_dose_cost(plan, Y, l, r):
    """cost [32] (float64) of 32 intensity vectors Y [N, 32] on fixed apertures."""
    N, R = plan.cfg.n_angles, plan.cfg.n_rows
    if Y.shape != (N, 32) or Y.dtype != torch.float32 or not Y.is_cuda:
        raise ValueError("Y must be a CUDA float32 tensor of shape [N, 32]")
    for t in (l, r):
        if t.dtype != torch.int16 or not t.is_cuda or t.numel() != N * R:
            raise ValueError("leaves must be CUDA int16 tensors of N*R entries")
    return _ApertureDoseCost.apply(Y, plan, l, r)
