"""torch.autograd.Function over the library: ell(X, Theta) with its adjoint.

The forward pass evaluates ell (Eq. (1)) together with d ell / d X (Appendix
A) and, when Theta requires a gradient, d ell / d Theta, in one call of the
C ABI; backward scales them by the incoming gradient.  Times get no
gradient.  Everything runs in the library's kernels.

    ll = hawkes_loglik_autograd(ctx, t, X, theta)   # theta: float64 tensor (6,)
    ll.backward()                                    # X.grad, theta.grad
"""
from __future__ import annotations

import torch

from .api import HawkesContext, hawkes_loglik_grad_locations


class HawkesLogLik(torch.autograd.Function):
    @staticmethod
    def forward(fctx, hctx: HawkesContext, t: torch.Tensor, X: torch.Tensor, theta: torch.Tensor,
                precision: str = "mixed"):
        want_theta = theta.requires_grad
        out = hawkes_loglik_grad_locations(hctx, t.detach(), X.detach(), theta.detach(), precision=precision,
                                           grad_params=want_theta)
        if want_theta:
            ell, gX, gT = out
        else:
            (ell, gX), gT = out, None
        fctx.save_for_backward(gX, gT if gT is not None else torch.empty(0, dtype=torch.float64,
                                                                            device=X.device))
        fctx.want_theta = want_theta
        return ell

    @staticmethod
    def backward(fctx, grad_out):
        gX, gT = fctx.saved_tensors
        dX = grad_out * gX if fctx.needs_input_grad[2] else None
        dT = grad_out * gT if (fctx.needs_input_grad[3] and fctx.want_theta) else None
        return None, None, dX, dT, None


def hawkes_loglik_autograd(ctx: HawkesContext, t: torch.Tensor, X: torch.Tensor, theta: torch.Tensor,
                           precision: str = "mixed") -> torch.Tensor:
    """ell as a differentiable 0-d tensor of X (N, D) and Theta (6,)."""
    if theta.dtype != torch.float64 or theta.numel() != 6:
        raise TypeError("theta must be a float64 tensor of the six parameters (mu0, tau_x, tau_t, theta, omega, h)")
    return HawkesLogLik.apply(ctx, t, X, theta, precision)
