"""torch.autograd.Function wrappers whose backward passes are the adjoint kernels.

PyTorch's convention for a real loss L of a complex tensor z is grad_z = dL/dRe z + i dL/dIm z.
With it:
  * Degrid  y = R s (Eq. rime), s real: grad_s = Re(R^H grad_y) = R^dagger grad_y, i.e. the
    gridding kernel without weights;
  * Grid    d = R^dagger (N^-1) y (Eq. clean): grad_y = N^-1 R grad_d (fr_degrid_weighted);
  * PsfLikelihood / ExactLikelihood  L_b = 1/2 s_b.(A s_b) - s_b.d_b with A = PSF * (Sec. 3.3.2)
    or R^dagger N^-1 R: grad_s = (A s - d) * grad_L (A is self-adjoint), grad_d = -s * grad_L.
    The forward kernel already produces A s - d, so backward costs no extra launch.
  * FastLikelihood  H_b = 1/2 r_b.(N'^-1 r_b), r = d - PSF * s (Eq. ham_new, Sec. 3.3.3, after
    Plan.noise_fit): grad_s = -PSF * (N'^-1 r) * grad_H and grad_d = N'^-1 r * grad_H (N'^-1
    symmetric); the forward kernel returns both vectors (fr_fast_likelihood_grad_resid).
All operator arithmetic runs in the library's CUDA kernels through binding.Plan; backward only
scales the saved vectors by the incoming gradient.
"""
from __future__ import annotations

import torch

from .binding import Plan


class Degrid(torch.autograd.Function):
    """R: sky [nsky, nx, ny] float32 -> vis [nrow, nchan] complex64."""

    @staticmethod
    def forward(ctx, sky, plan):
        ctx.plan = plan
        return plan.degrid(sky.contiguous())

    @staticmethod
    def backward(ctx, grad_vis):
        return ctx.plan.grid(grad_vis.contiguous(), apply_weights=False), None


class Grid(torch.autograd.Function):
    """R^dagger (N^-1): vis [nrow, nchan] complex64 -> [nsky, nx, ny] float32."""

    @staticmethod
    def forward(ctx, vis, plan, apply_weights=True):
        ctx.plan = plan
        ctx.apply_weights = apply_weights
        return plan.grid(vis.contiguous(), apply_weights=apply_weights)

    @staticmethod
    def backward(ctx, grad_dirty):
        return ctx.plan.degrid(grad_dirty.contiguous(), weighted=ctx.apply_weights), None, None


class PsfLikelihood(torch.autograd.Function):
    """L_b = 1/2 s_b.(PSF * s_b) - s_b.d_b for sky, dirty [batch, nsky, nx, ny]; returns [batch]."""

    @staticmethod
    def forward(ctx, sky, dirty, plan, exact=False):
        value, grad = plan.likelihood_grad(sky.contiguous(), dirty.contiguous(), exact=exact)
        ctx.save_for_backward(sky, grad)
        return torch.as_tensor(value, dtype=torch.float64, device=sky.device)

    @staticmethod
    def backward(ctx, grad_value):
        sky, grad = ctx.saved_tensors
        gv = grad_value.to(torch.float32).view(-1, *([1] * (sky.dim() - 1)))
        gs = grad * gv if ctx.needs_input_grad[0] else None
        gd = -sky * gv if ctx.needs_input_grad[1] else None
        return gs, gd, None, None


class FastLikelihood(torch.autograd.Function):
    """H_b of Eq. ham_new for sky, dirty [batch, nsky, nx, ny] (or [nsky, nx, ny]); returns [batch]."""

    @staticmethod
    def forward(ctx, sky, dirty, plan):
        if ctx.needs_input_grad[1]:
            value, grad, nr = plan.fast_likelihood_grad(sky.contiguous(), dirty.contiguous(),
                                                        want_ninv_resid=True)
        else:
            value, grad = plan.fast_likelihood_grad(sky.contiguous(), dirty.contiguous())
            nr = None
        ctx.save_for_backward(sky, grad, nr)
        return torch.as_tensor(value, dtype=torch.float64, device=sky.device)

    @staticmethod
    def backward(ctx, grad_value):
        sky, grad, nr = ctx.saved_tensors
        gv = grad_value.to(torch.float32).view(-1, *([1] * (sky.dim() - 1)))
        if sky.dim() == 3:
            gv = gv.view(*([1] * sky.dim()))
        gs = grad * gv if ctx.needs_input_grad[0] else None
        gd = nr * gv if ctx.needs_input_grad[1] else None
        return gs, gd, None


def degrid(sky, plan):
    return Degrid.apply(sky, plan)


def grid(vis, plan, apply_weights=True):
    return Grid.apply(vis, plan, apply_weights)


def psf_likelihood(sky, dirty, plan):
    return PsfLikelihood.apply(sky, dirty, plan, False)


def exact_likelihood(sky, dirty, plan):
    return PsfLikelihood.apply(sky, dirty, plan, True)


def fast_likelihood(sky, dirty, plan):
    return FastLikelihood.apply(sky, dirty, plan)
