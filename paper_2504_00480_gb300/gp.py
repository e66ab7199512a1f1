"""Additive-kernel GP training and prediction on top of the C ABI (Sec. 5).

The hyperparameters (ell, sigma_f, sigma_eps) are trained in R and mapped to
the kernel through softplus (Sec. 5); Adam (learning rate 0.01) follows the
gradient of the NLML estimate of Sec. 1, computed by ``agp_nlml_grad`` (M =
I) or ``agp_nlml_grad_pc`` (landmark preconditioner, Sec. 2.3). Prediction
solves K_hat alpha = y by (P)CG and applies the cross kernel K(X*, X) alpha as
the test rows of one matvec over the union of training and test points, with
the training block of the input set to alpha and the test block to zero (no
noise term). Every matvec, solve and gradient runs in the library's kernels;
this module only holds the optimiser state and the loop.

Defaults follow Sec. 5: 500 Adam iterations, 10 probes and 10 Lanczos
steps per gradient, 10 landmarks per feature window, 50 CG iterations for
prediction.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import agp


def softplus(x: np.ndarray) -> np.ndarray:
    return np.logaddexp(0.0, x)


def softplus_grad(x: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + np.tanh(0.5 * x))   # the logistic function, overflow-free


class AdditiveGP:
    """GP regression with the additive kernel K_hat = sigma_f^2 sum_s K_s +
    sigma_eps^2 I over feature windows (Sec. 2.1), applied through the
    library's NFFT fast summation.

    X: (n, p) array already scaled into [-1/4, 1/4) (Sec. 3.1); y: (n,)."""

    def __init__(self, X, y, windows, kernel: str = "gauss", N=32, cutoff: int = 5,
                 dtype=torch.float32, raw_init=(0.0, 0.0, 0.0), device: str = "cuda:0",
                 landmarks_per_window: int = 10):
        self.X = np.asarray(X, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64).reshape(-1)
        self.windows = [list(w) for w in windows]
        self.kernel, self.N, self.cutoff = kernel, N, cutoff
        self.dtype, self.device = dtype, device
        self.raw = np.asarray(raw_init, dtype=np.float64).copy()
        self.n_landmarks = min(480, landmarks_per_window * len(self.windows))
        ell, sf, se = self.hyper()
        self.plan = agp.Plan(torch.tensor(self.X, dtype=dtype, device=device), self.windows,
                             N, cutoff, kernel, ell, sf, se)
        self.yt = torch.tensor(self.y, dtype=dtype, device=device)
        self._m = np.zeros(3)
        self._v = np.zeros(3)
        self._t = 0

    def hyper(self):
        """(ell, sigma_f, sigma_eps) = softplus(raw)."""
        return tuple(float(v) for v in softplus(self.raw))

    def nlml_and_grad(self, n_probes: int = 10, lanczos_steps: int = 10, seed: int = 0,
                      preconditioned: bool = True):
        """NLML estimate and its gradient with respect to the raw parameters
        (chain rule through softplus)."""
        ell, sf, se = self.hyper()
        self.plan.set_hyper(ell, sf, se)
        n = self.X.shape[0]
        rng = np.random.default_rng(seed)
        if preconditioned:
            k = len(self.plan.landmarks(self.n_landmarks))
            Wn = torch.tensor(rng.standard_normal((n, n_probes)), dtype=self.dtype,
                              device=self.device)
            Wk = rng.standard_normal((k, n_probes))
            nl, g = self.plan.nlml_grad_pc(self.yt, Wn, Wk, self.n_landmarks,
                                           lanczos_steps=lanczos_steps)
        else:
            Z = torch.tensor(rng.integers(0, 2, (n, n_probes)) * 2.0 - 1.0, dtype=self.dtype,
                             device=self.device)
            nl, g = self.plan.nlml_grad(self.yt, Z, lanczos_steps=lanczos_steps)
        grad_theta = np.array([g["ell"], g["sigma_f"], g["sigma_eps"]])
        return nl, grad_theta * softplus_grad(self.raw)

    def step(self, lr: float = 0.01, **kw):
        """One Adam step (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the NLML."""
        nl, g = self.nlml_and_grad(**kw)
        self._t += 1
        self._m = 0.9 * self._m + 0.1 * g
        self._v = 0.999 * self._v + 0.001 * g * g
        mh = self._m / (1.0 - 0.9 ** self._t)
        vh = self._v / (1.0 - 0.999 ** self._t)
        self.raw = self.raw - lr * mh / (np.sqrt(vh) + 1e-8)
        return nl

    def fit(self, iters: int = 500, lr: float = 0.01, n_probes: int = 10,
            lanczos_steps: int = 10, preconditioned: bool = True, seed: int = 0):
        """Adam on the NLML estimate; returns the NLML estimate of every step."""
        hist = []
        for it in range(iters):
            hist.append(self.step(lr, n_probes=n_probes, lanczos_steps=lanczos_steps,
                                  seed=seed + it, preconditioned=preconditioned))
        ell, sf, se = self.hyper()
        self.plan.set_hyper(ell, sf, se)
        return hist

    def predict(self, X_test, cg_iters: int = 50, rtol: float = 0.0,
                preconditioned: bool = True):
        """Posterior mean K(X*, X) K_hat^{-1} y (Sec. 5: 50 CG iterations)."""
        ell, sf, se = self.hyper()
        self.plan.set_hyper(ell, sf, se)
        alpha, _, _ = self.plan.solve(self.yt[:, None].contiguous(), rtol=rtol, maxit=cg_iters,
                                      raise_not_converged=False,
                                      n_landmarks=self.n_landmarks if preconditioned else 0)
        Xs = np.asarray(X_test, dtype=np.float64)
        union = np.concatenate([self.X, Xs], axis=0)
        up = agp.Plan(torch.tensor(union, dtype=self.dtype, device=self.device), self.windows,
                      self.N, self.cutoff, self.kernel, ell, sf, se)
        V = torch.zeros((union.shape[0], 1), dtype=self.dtype, device=self.device)
        V[: self.X.shape[0]] = alpha
        out = up.matvec(V, add_noise=False)
        up.close()
        return out[self.X.shape[0]:, 0].cpu().numpy().astype(np.float64)


__all__ = ["AdditiveGP", "softplus", "softplus_grad"]
