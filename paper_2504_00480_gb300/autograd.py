"""torch.autograd.Function over the library's additive-kernel matvec.

Forward:  Out = K_hat(theta) V,  theta = (ell, sigma_f, sigma_eps)  (Sec. 2.1),
          through agp_matvec_spectra, which also keeps the forward spectra of
          V (spread + DFT, before deconvolution) for the backward pass.
Backward, for an upstream gradient G (every product runs in libagp.so):
  dL/dV         = K_hat G            (K_hat is symmetric: the library outputs the
                                      real part of eq. (3.3), a symmetric operator)
  dL/dell       = sum_r G_r^T (sigma_f^2 sum_s K_s^der V_r)
                = sigma_f^2 sum_s sum_k D^der_k Re(conj(g_k) v_k)
                  (Sec. 3.2 eq. (3.4): the derivative sits on the Fourier
                  coefficients, so only the spectra g of G are formed -- one
                  spread and one forward DFT -- and paired with V's)
  dL/dsigma_f   = sum_r G_r^T (2 sigma_f sum_s K_s V_r)
                = 2 sigma_f sum_s sum_k D_k Re(conj(g_k) v_k)   (same spectra)
  dL/dsigma_eps = sum_r G_r^T 2 sigma_eps V_r
When V needs a gradient the spectra of G come out of the K_hat G matvec at no
extra cost. The sigma_eps term is an FP64 column dot product of the library. The
plan's coefficients are recomputed only if its hyperparameters changed
between forward and backward. After the backward the library's timeout flag
is checked (AGP_TIMEOUT raises). This is the derivative the hyperparameter
training of Sec. 1 needs: d(v^T K_hat w)/d(v, w, theta) follows from
(v * matvec(w)).sum().
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
        plan.ensure_hyper(*theta)
        V2 = V if V.dim() == 2 else V.unsqueeze(1)
        V2 = V2.contiguous()
        out, spec = plan.spectra(V2, out=True)
        ctx.plan = plan
        ctx.theta = theta
        ctx.vdim = V.dim()
        ctx.save_for_backward(V2, spec)
        return out if V.dim() == 2 else out.squeeze(1)

    @staticmethod
    def backward(ctx, G):
        V, specV = ctx.saved_tensors
        plan = ctx.plan
        ell, sf, se = ctx.theta
        plan.ensure_hyper(ell, sf, se)
        G2 = (G if G.dim() == 2 else G.unsqueeze(1)).contiguous()
        R = G2.shape[1]
        gV = g_ell = g_sf = g_se = None
        dt = torch.float64
        if any(ctx.needs_input_grad[:3]):
            gV, specG = plan.spectra(G2, out=True if ctx.needs_input_grad[0] else None)
            if gV is not None and ctx.vdim == 1:
                gV = gV.squeeze(1)
            if ctx.needs_input_grad[1]:
                g_ell = plan.spectral_form("ell", specG, specV, R).sum().cpu().to(dt)
            if ctx.needs_input_grad[2]:
                g_sf = plan.spectral_form("sigma_f", specG, specV, R).sum().cpu().to(dt)
        if ctx.needs_input_grad[3]:
            g_se = torch.tensor(2.0 * se * _dot(plan, G2, V), dtype=dt)
        plan.check()
        return gV, g_ell, g_sf, g_se, None


def additive_kernel_matvec(plan, V, ell, sigma_f, sigma_eps):
    """Differentiable Out = K_hat V. ell, sigma_f, sigma_eps: python floats or
    0-dim tensors (float64 tensors with requires_grad receive gradients)."""
    def t(x):
        return x if torch.is_tensor(x) else torch.tensor(float(x), dtype=torch.float64)
    return AdditiveKernelMatvec.apply(V, t(ell), t(sigma_f), t(sigma_eps), plan)
