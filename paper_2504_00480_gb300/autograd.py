"""torch.autograd.Function over the library's additive-kernel matvec.

Forward:  Out = K_hat(theta) V,  theta = (ell, sigma_f, sigma_eps)  (Sec. 2.1).
Backward, for an upstream gradient G (all products run in libagp.so):
  dL/dV         = K_hat G            (K_hat is symmetric: the library outputs the
                                      real part of eq. (3.3), a symmetric operator)
  dL/dell       = sum_r G_r^T (sigma_f^2 sum_s K_s^der V_r)   (eq. (2.3) with the
                                      derivative-kernel coefficients, Sec. 3.2)
  dL/dsigma_f   = sum_r G_r^T (2/sigma_f) (Out_r - sigma_eps^2 V_r)
  dL/dsigma_eps = sum_r G_r^T 2 sigma_eps V_r
The column dot products are FP64 reductions of the library (agp_dot_columns).
This is the derivative the hyperparameter training of Sec. 1 needs:
d(v^T K_hat w)/d(v, w, theta) follows from (v * matvec(w)).sum().
"""
from __future__ import annotations

import torch

from . import agp


def _dot(plan, A, B):
    return float(agp.agp_dot_columns(plan.handle, A, B).sum())


class AdditiveKernelMatvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, ell, sigma_f, sigma_eps, plan):
        theta = (float(ell), float(sigma_f), float(sigma_eps))
        plan.set_hyper(*theta)
        V2 = V if V.dim() == 2 else V.unsqueeze(1)
        V2 = V2.contiguous()
        out = plan.matvec(V2)
        ctx.plan = plan
        ctx.theta = theta
        ctx.vdim = V.dim()
        ctx.save_for_backward(V2, out)
        return out if V.dim() == 2 else out.squeeze(1)

    @staticmethod
    def backward(ctx, G):
        V, out = ctx.saved_tensors
        plan = ctx.plan
        ell, sf, se = ctx.theta
        plan.set_hyper(ell, sf, se)
        G2 = (G if G.dim() == 2 else G.unsqueeze(1)).contiguous()
        gV = g_ell = g_sf = g_se = None
        if ctx.needs_input_grad[0]:
            gV = plan.matvec(G2)
            if ctx.vdim == 1:
                gV = gV.squeeze(1)
        dt = torch.float64
        if ctx.needs_input_grad[1]:
            g_ell = torch.tensor(_dot(plan, G2, plan.deriv_matvec("ell", V)), dtype=dt)
        if ctx.needs_input_grad[2]:
            if sf != 0.0:   # (2/sigma_f) (G.Out - sigma_eps^2 G.V): no extra matvec
                g = (2.0 / sf) * (_dot(plan, G2, out) - se * se * _dot(plan, G2, V))
            else:
                g = _dot(plan, G2, plan.deriv_matvec("sigma_f", V))
            g_sf = torch.tensor(g, dtype=dt)
        if ctx.needs_input_grad[3]:
            g_se = torch.tensor(2.0 * se * _dot(plan, G2, V), dtype=dt)
        return gV, g_ell, g_sf, g_se, None


def additive_kernel_matvec(plan, V, ell, sigma_f, sigma_eps):
    """Differentiable Out = K_hat V. ell, sigma_f, sigma_eps: python floats or
    0-dim tensors (float64 tensors with requires_grad receive gradients)."""
    def t(x):
        return x if torch.is_tensor(x) else torch.tensor(float(x), dtype=torch.float64)
    return AdditiveKernelMatvec.apply(V, t(ell), t(sigma_f), t(sigma_eps), plan)
