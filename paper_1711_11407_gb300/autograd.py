"""Differentiable line projection and sparse synthesis, and least-squares amplitude refinement.

Both maps of FPS-SFT are linear in their complex input:
  P: cube x -> line bins, the L-point DFTs of the D+1 lines of every schedule row (Eq. sample_slice,
     Eq. hs);
  S: amplitudes a -> line bins of the sparse spectrum {(k_i, a_i)} (Eq. freqSum), for a fixed support.
For a linear map y = A x, PyTorch's backward for complex tensors returns A^H g for the incoming
gradient g; the adjoint kernels of the library compute exactly P^H g (inverse-direction DFT and
scatter-add) and S^H g (gather-reduce), so these Functions differentiate through the CUDA path.

`refine` re-estimates the amplitudes of a recovered support by least squares over many lines:
minimise sum_rows ||P x - S a||^2 over a (per signal), by conjugate gradients on the normal
equations S^H S a = S^H P x, whose operator the library applies in one fused kernel (S and S^H
through shared-memory bins).  The decode uses one bin of one line per frequency (Eq. decoding);
the refinement averages the noise over every line of the schedule.
"""
from __future__ import annotations

import torch

from .api import Plan

__all__ = ["LineProject", "SparseSynth", "line_project", "sparse_synth", "refine"]


class LineProject(torch.autograd.Function):
    """cubes (complex64, flat, signals at `offsets`) -> bins [batch][n_sched][D+1][L_max]."""

    @staticmethod
    def forward(ctx, cubes, plan: Plan, offsets, alpha, tau):
        ctx.plan = plan
        ctx.numel = cubes.numel()
        ctx.save_for_backward(offsets, alpha, tau)
        return plan.project(cubes.contiguous(), offsets, alpha, tau)

    @staticmethod
    def backward(ctx, grad_bins):
        offsets, alpha, tau = ctx.saved_tensors
        g = torch.zeros(ctx.numel, dtype=torch.complex64, device=grad_bins.device)
        ctx.plan.adjoint_project(grad_bins.contiguous(), offsets, alpha, tau, g)
        return g, None, None, None, None


class SparseSynth(torch.autograd.Function):
    """amplitudes a [batch][k_cap] (entries i < count[b] used) -> bins [batch][n_sched][D+1][L_max]."""

    @staticmethod
    def forward(ctx, a, plan: Plan, k, count, alpha, tau):
        ctx.plan = plan
        ctx.save_for_backward(k, count, alpha, tau)
        return plan.synth(alpha, tau, k, a.contiguous(), count)

    @staticmethod
    def backward(ctx, grad_bins):
        k, count, alpha, tau = ctx.saved_tensors
        ga = torch.zeros((ctx.plan.batch, ctx.plan.k_cap), dtype=torch.complex64, device=grad_bins.device)
        ctx.plan.adjoint_synth(grad_bins.contiguous(), alpha, tau, k, count, ga)
        return ga, None, None, None, None, None


def line_project(cubes, plan, offsets, alpha, tau):
    return LineProject.apply(cubes, plan, offsets, alpha, tau)


def sparse_synth(a, plan, k, count, alpha, tau):
    return SparseSynth.apply(a, plan, k, count, alpha, tau)


def refine(plan: Plan, cubes, offsets, k, a0, count, alpha, tau, iters=25, tol=1e-7, stream=None):
    """Least-squares amplitudes on a fixed support, per signal: argmin_a sum ||P x - S a||^2 over the
    schedule rows alpha/tau [batch][n_sched][D].  The line DFTs P x come from the projection kernel
    and the conjugate-gradient loop runs in the library (fpssft_refine: two launches per iteration,
    no host synchronisation, so the call can sit inside a captured CUDA graph).
    Returns (a, residual norms ||P x - S a|| per signal)."""
    y = plan.project(cubes, offsets, alpha, tau, stream=stream)
    a = a0.detach().clone()
    return plan.refine(y, alpha, tau, k, a, count, iters=iters, tol=tol, stream=stream)
