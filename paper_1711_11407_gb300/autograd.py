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
equations, with S a from the synthesis kernel and S^H r from its autograd backward.  The decode
uses one bin of one line per frequency (Eq. decoding); the refinement averages the noise over
every line of the schedule.
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


def _adjoint_synth(plan, k, count, alpha, tau, r):
    """S^H r through the autograd backward of SparseSynth."""
    a = torch.zeros((plan.batch, plan.k_cap), dtype=torch.complex64, device=r.device, requires_grad=True)
    y = sparse_synth(a, plan, k, count, alpha, tau)
    (g,) = torch.autograd.grad(y, a, grad_outputs=r)
    return g


def refine(plan: Plan, cubes, offsets, k, a0, count, alpha, tau, iters=25, tol=1e-7):
    """Least-squares amplitudes on a fixed support, per signal: argmin_a sum ||P x - S a||^2 over the
    schedule rows alpha/tau [batch][n_sched][D].  Returns (a, residual norms per signal)."""
    mask = (torch.arange(plan.k_cap, device=a0.device)[None, :] < count[:, None].long())
    y = line_project(cubes, plan, offsets, alpha, tau).detach()
    a = (a0 * mask).detach().clone()

    def S(v):
        return sparse_synth(v, plan, k, count, alpha, tau).detach()

    def dot(u, v):       # per-signal <u, v> over all but the batch axis
        return torch.sum((u.conj() * v).reshape(u.shape[0], -1), dim=1)

    r = _adjoint_synth(plan, k, count, alpha, tau, y - S(a)) * mask       # S^H (y - S a)
    p = r.clone()
    rr = dot(r, r).real
    rr0 = rr.clone()
    for _ in range(iters):
        q = S(p)
        qq = dot(q, q).real
        step = torch.where(qq > 0, rr / torch.clamp(qq, min=1e-30), torch.zeros_like(qq))
        a = a + step[:, None] * p
        r = r - step[:, None] * (_adjoint_synth(plan, k, count, alpha, tau, q) * mask)
        rr_new = dot(r, r).real
        beta = torch.where(rr > 0, rr_new / torch.clamp(rr, min=1e-30), torch.zeros_like(rr))
        p = r + beta[:, None] * p
        rr = rr_new
        if bool(torch.all(rr <= tol * tol * torch.clamp(rr0, min=1e-30))):
            break
    res = torch.sqrt(dot(y - S(a), y - S(a)).real)
    return a.detach(), res
