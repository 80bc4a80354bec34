"""Differentiable Vegas estimate of the Eq. 1 Gaussian integral.

``gauss_integral(mu, a, vegas, it, n)`` returns the fixed-grid estimate
I(mu, a) = (1/n) sum_i f(x_i; mu, a) J_i over samples 0..n-1 of iteration
``it`` on ``vegas``'s current grid, as a 0-d tensor that autograd can
differentiate in mu (shape [d]) and a.  Forward and backward each call the
CUDA adjoint kernel (vegas_gauss_adjoint), which regenerates the samples from
their counters: nothing per sample is kept between the two passes.  On a
frozen grid the samples do not depend on (mu, a), so the backward pass gives
the exact derivative of the estimate (the reparameterised estimator).
"""
import torch

from .binding import vegas_gauss_adjoint


class GaussIntegral(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, a, vegas, it, n):
        d = vegas.dim
        params = [float(a)] + [float(v) for v in mu.detach().reshape(-1).cpu().tolist()]
        if len(params) != d + 1:
            raise ValueError(f"mu must have {d} entries")
        out = torch.empty(2 * (d + 2) + 1, dtype=torch.float64, device=vegas.workspace.device)
        vegas_gauss_adjoint(vegas.handle, params, it, n, 0, out.data_ptr())
        ctx.vegas, ctx.it, ctx.n, ctx.params = vegas, it, n, params
        ctx.mu_meta = (mu.shape, mu.dtype, mu.device)
        ctx.a_meta = (a.shape, a.dtype, a.device)
        return out[0].clone()

    @staticmethod
    def backward(ctx, grad_out):
        v = ctx.vegas
        d = v.dim
        out = torch.empty(2 * (d + 2) + 1, dtype=torch.float64, device=v.workspace.device)
        vegas_gauss_adjoint(v.handle, ctx.params, ctx.it, ctx.n, 1, out.data_ptr())
        g = grad_out.to(torch.float64)
        shape, dtype, device = ctx.mu_meta
        gmu = (out[1:d + 1] * g).reshape(shape).to(device=device, dtype=dtype)
        ashape, adtype, adevice = ctx.a_meta
        ga = (out[d + 1] * g).reshape(ashape).to(device=adevice, dtype=adtype)
        return gmu, ga, None, None, None


def gauss_integral(mu, a, vegas, it, n):
    """Differentiable I(mu, a); see the module docstring."""
    return GaussIntegral.apply(mu, a, vegas, it, n)
