"""Seeded synthetic inputs for the additive-kernel fast summation.

This module only draws and scales random numbers. It holds none of the
method's arithmetic (no kernel, no Fourier coefficient, no window function),
so both the CUDA path and the CPU oracle can be fed from it.

Every generator uses ``numpy.random.default_rng(seed)``. Points are min-max
scaled per feature into [-0.24, 0.24], which lies inside the box
[-1/4, 1/4)^d that the paper scales each feature window into (Sec. 3.1).

The five workloads follow the paper's experimental shapes and the five
configurations this library is benchmarked on:

* ``plain_fp64``      n=1,000, p=2, one d=2 window, Gaussian ell=0.3, N=32, s=4
* ``autograd``        n=100,000, p=9, three d=3 windows, Gaussian ell=0.2, N=32, s=5
* ``batched_pcg``     n=500,000, p=12 uniform, four d=3 windows, Matern(1/2) ell=0.5
* ``nlml_grad``       n=1,000,000, p=8, windows d=(3,3,2), Gaussian, N=32/64, s=5
* ``uneven_batch``    64 problems, n log-uniform in [1e4, 2e5], p=6, two d=3 windows

Window feature indices are 0-based (the paper prints them 1-based).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LO, HI = -0.24, 0.24


def minmax_scale(X: np.ndarray, lo: float = LO, hi: float = HI) -> np.ndarray:
    """Affine per-feature map of the data range onto [lo, hi] (float64)."""
    X = np.asarray(X, dtype=np.float64)
    mn = X.min(axis=0, keepdims=True)
    mx = X.max(axis=0, keepdims=True)
    span = np.where(mx > mn, mx - mn, 1.0)
    Y = lo + (hi - lo) * (X - mn) / span
    return np.clip(Y, lo, hi)


def ball_scale(X: np.ndarray, windows, radius: float) -> np.ndarray:
    """Scale each window's columns (already centred, e.g. by minmax_scale) by
    one factor so that the largest Euclidean norm of a window point is
    ``radius`` (float64)."""
    Y = np.array(X, dtype=np.float64)
    for w in windows:
        cols = list(w)
        m = np.sqrt((Y[:, cols] ** 2).sum(axis=1)).max()
        if m > 0:
            Y[:, cols] *= radius / m
    return Y


def standardize(X: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    sd = X.std(axis=0, keepdims=True)
    return (X - X.mean(axis=0, keepdims=True)) / np.where(sd > 0, sd, 1.0)


def to_precision(X: np.ndarray, dtype) -> np.ndarray:
    """Round the scaled points to the working precision.

    The CUDA path and the oracle then see the same point values: the oracle
    upcasts these rounded values to float64."""
    Y = np.asarray(X, dtype=dtype)
    # Rounding cannot leave [-1/4, 1/4): |x| <= 0.24 before rounding.
    return Y


def rademacher(n: int, R: int, seed: int) -> np.ndarray:
    """n x R matrix of independent +-1 entries (Hutchinson probes, Sec. 1)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(n, R)).astype(np.float64) * 2.0 - 1.0


def gaussian(m: int, R: int, seed: int) -> np.ndarray:
    """m x R matrix of independent standard normal entries (the vectors w
    from which the preconditioned likelihood builds its probes)."""
    return np.random.default_rng(seed).standard_normal((m, R))


@dataclass
class Workload:
    name: str
    X: np.ndarray                 # (n, p) scaled points, float64 holding `dtype` values
    windows: list                 # list of lists of 0-based feature ids
    kernel: str                   # "gauss" | "matern12" | "matern32" | "imq" | "sinc"
    ell: float
    sigma_f: float
    sigma_eps: float
    N: list                       # Fourier bandwidth per window (paper's m)
    cutoff: int                   # window half-support s
    dtype: type = np.float32
    V: np.ndarray | None = None   # (n, R) right-hand sides
    y: np.ndarray | None = None   # labels, where the workload has them
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.X.shape[0]


def _points(X, dtype):
    return to_precision(minmax_scale(X), dtype).astype(np.float64)


def plain_fp64(n: int = 1000, seed: int = 0) -> Workload:
    """Plain method in FP64: p=2 features from N(0,1), one window {0,1}."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 2))
    V = rng.standard_normal((n, 1))
    return Workload("plain_fp64", _points(X, np.float64), [[0, 1]], "gauss",
                    0.3, 1.0, 0.0, [32], 4, np.float64, V=V)


def autograd(n: int = 100_000, seed: int = 1, R: int = 1) -> Workload:
    """p=9 standardized Gaussian features, windows {0,1,2},{3,4,5},{6,7,8}."""
    rng = np.random.default_rng(seed)
    X = standardize(rng.standard_normal((n, 9)))
    V = rng.standard_normal((n, R))
    W = rng.standard_normal((n, R))
    return Workload("autograd", _points(X, np.float32),
                    [[0, 1, 2], [3, 4, 5], [6, 7, 8]], "gauss",
                    0.2, 1.0, 0.1, [32, 32, 32], 5, np.float32, V=V,
                    extra={"W": W})


def batched_pcg(n: int = 500_000, seed: int = 2, R: int = 32, ell: float = 0.5,
                N: int = 64) -> Workload:
    """p=12 uniform[-1,1] features, four consecutive d=3 windows, Matern(1/2).

    Labels y = sum_w sin(2 pi x_w1) cos(pi x_w2) x_w3 + N(0, 0.05^2) on the raw
    features; right-hand sides [y, R-1 Rademacher probes]. Grid N = 64 per
    dimension by default: at N = 32 the Fourier-truncated Matern operator
    with ell = 0.5 has negative coefficients that make K_hat indefinite on
    this point set already at n = 20,000 (CG diverges in FP64). ``ell`` and
    ``N`` select a variant (the truncated series has no negative coefficient
    for ell <= 0.09 at N = 32)."""
    rng = np.random.default_rng(seed)
    raw = rng.uniform(-1.0, 1.0, size=(n, 12))
    windows = [[0, 1, 2], [3, 4, 5], [6, 7, 8], [9, 10, 11]]
    y = np.zeros(n)
    for w in windows:
        y += np.sin(2 * np.pi * raw[:, w[0]]) * np.cos(np.pi * raw[:, w[1]]) * raw[:, w[2]]
    y += 0.05 * rng.standard_normal(n)
    V = np.concatenate([y[:, None], rademacher(n, R - 1, seed + 100)], axis=1)
    return Workload("batched_pcg", _points(raw, np.float32), windows, "matern12",
                    float(ell), 1.0, 0.05, [int(N)] * 4, 5, np.float32, V=V, y=y)


def nlml_grad(n: int = 1_000_000, seed: int = 3, R: int = 32) -> Workload:
    """p=8 standardized Gaussian features, windows {0,1,2},{3,4,5},{6,7}.

    sigma_f = sigma_eps = softplus(0) = ln 2 (the paper's initial point);
    ell = 0.1: at ell = ln 2 the Fourier-truncated Gaussian has negative
    coefficients (down to -1e-2 of the largest) that make K_hat indefinite at
    n = 1e6, so the log-determinant of the likelihood is undefined; at 0.1
    the most negative coefficient is ~6e-9 and K_hat stays positive definite.
    Labels y = sum_w sin(2 pi x_w1) cos(pi x_w2) + N(0, 0.1^2) on the raw
    features; right-hand sides [y, R-1 Rademacher probes]."""
    rng = np.random.default_rng(seed)
    raw = standardize(rng.standard_normal((n, 8)))
    windows = [[0, 1, 2], [3, 4, 5], [6, 7]]
    y = np.zeros(n)
    for w in windows:
        y += np.sin(2 * np.pi * raw[:, w[0]] / 4) * np.cos(np.pi * raw[:, w[1]] / 4)
    y += 0.1 * rng.standard_normal(n)
    V = np.concatenate([y[:, None], rademacher(n, R - 1, seed + 100)], axis=1)
    ln2 = math.log(2.0)
    return Workload("nlml_grad", _points(raw, np.float32), windows, "gauss",
                    0.1, ln2, ln2, [32, 32, 64], 5, np.float32, V=V, y=y)


def uneven_batch(n_problems: int = 64, seed: int = 4, n_lo: int = 10_000,
                 n_hi: int = 200_000, R: int = 1):
    """Independent problems with n log-uniform in [n_lo, n_hi], p=6, two d=3
    windows, per-problem Gaussian lengthscale uniform in [0.1, 0.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_problems):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        X = rng.standard_normal((n, 6))
        ell = float(rng.uniform(0.1, 0.5))
        V = rng.standard_normal((n, R))
        out.append(Workload(f"uneven_batch[{q}]", _points(X, np.float32),
                            [[0, 1, 2], [3, 4, 5]], "gauss", ell, 1.0, 0.1,
                            [32, 32], 4, np.float32, V=V))
    return out


def subset(w: Workload, n: int) -> Workload:
    """First n points of a workload (same windows and hyperparameters)."""
    import copy
    c = copy.copy(w)
    c.X = w.X[:n]
    c.V = None if w.V is None else w.V[:n]
    c.y = None if w.y is None else w.y[:n]
    c.extra = {k: (v[:n] if isinstance(v, np.ndarray) else v) for k, v in w.extra.items()}
    c.name = f"{w.name}[:{n}]"
    return c
