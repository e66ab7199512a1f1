"""Plain, slow FP64 reference of the additive-kernel fast summation.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Paper: "Preconditioned Additive Gaussian Processes with Fourier Acceleration"
(arXiv 2504.00480). Every function names the passage it follows. Where the
paper is silent or ambiguous this module takes the following readings:

* The paper's bandwidth m is called ``N`` here; ``I_N = {-N/2, ..., N/2-1}^d``.
* The fast sum outputs the REAL part of eq. (3.3); with the asymmetric index
  set the complex sum has a small imaginary part, and the paper's own 1-D
  figure (Sec. 3.1) shows the real cosine series.
* ``kappa_R(l/N)`` at ``l_t = -N/2`` is the plain kernel value (no boundary
  smoothing, Sec. 3.1), unless outer boundary smoothing is asked for
  (``boundary = (eps_b, p)``): then kappa_R follows the two-point Taylor
  regularisation of ``boundary_polynomial``, whose value at r = 1/2 is
  kappa(1/2).
* One lengthscale and one ``sigma_f`` are shared by all windows (Sec. 2.1).
* NFFT (Appendix A): Kaiser-Bessel window with oversampling ``sigma_os``
  (default 2, so the oversampled grid has ``n_os = 2N`` points per dimension).
  Its Fourier transform is the standard closed form in the modified Bessel
  function I0, which the paper mentions but does not print.

Pins (tests/test_oracle_*.py, all ``-m "not gpu"``):

* ``kernel``/``kernel_der_ell``: textbook values, finite differences in ell.
* ``dense_matvec``: brute-force double loop on tiny n, identical points
  (closed form), translation invariance, symmetry, positive definiteness.
* ``fourier_coeffs``: the paper's worked example (1-D Matern, ell=0.3, N=8,
  golden file), the geometric-series closed form of 1-D Matern, the Gaussian
  Fourier transform at small ell, separability of the Gaussian.
* ``truncated_matvec``: exact agreement with the dense sum on lattice points
  (trigonometric interpolation property), convergence to the dense sum at
  small ell, exact symmetry, eq. (3.4) derivative consistency.
* ``kernel_taylor``: symbolic derivatives (sympy); ``boundary_polynomial``:
  the 2p interpolation conditions checked by finite differences of the
  regularised kernel, continuity of kappa_R's derivatives; the smoothed
  truncated sum converges to the dense sum faster than the unsmoothed one
  (Gaussian, Matern(3/2)), and eq. (3.4) derivative consistency holds with
  smoothing.
* ``kb_window_hat``: numerical quadrature of the truncated window.
* ``nfft``/``nfft_adjoint``: error against the exact NDFT below the window
  error bound of Appendix A.
* ``afn_*``/``fsai_pattern``: the FSAI factor with a full pattern equals the
  inverse Cholesky factor of the Schur complement and M equals K_hat; the
  FSAI defining equations; M's landmark rows equal K_hat's; fill 1 keeps
  K_hat's diagonal; dense solve and slogdet; finite differences of log det M,
  of G and of M; Z Z^T = M for the probes of the identity; the AFN likelihood
  estimate is exact with a full pattern and equals the dense Hutchinson
  average with a full Krylov space.
* ``cg``: dense Cholesky solve; ``slq_quadratic``: eigendecomposition-based
  matrix logarithm with full Krylov space, and at the Lanczos breakdown floor
  (``LANCZOS_BREAKDOWN``) well before it; ``nlml_exact``: scipy's
  multivariate normal log density.
* ``splitmix64``/``rademacher_probes``: the generator's published output
  values; ``farthest_point_sampling``/``fsai_pattern``: brute-force FP64
  distances on small sets.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

__all__ = [
    "kernel", "kernel_der_ell", "window_points",
    "dense_matvec", "dense_deriv_matvec", "dense_matrix",
    "kernel_taylor", "boundary_polynomial", "kernel_regularised",
    "index_set", "fourier_coeffs", "ndft_adjoint", "ndft",
    "truncated_matvec", "truncated_deriv_matvec", "truncated_operators", "truncated_forms",
    "bins", "kb_shape", "kb_window", "kb_window_hat",
    "nfft_adjoint", "nfft", "nfft_fastsum_matvec",
    "cg", "pcg", "LANCZOS_BREAKDOWN", "farthest_point_sampling", "farthest_point_gaps", "additive_landmarks",
    "nystrom_preconditioner",
    "splitmix64", "rademacher_probes", "lanczos_tridiag_from_cg", "slq_quadratic",
    "nlml_exact", "nlml_estimate",
    "landmark_jitter", "nystrom_blocks", "nystrom_matrix", "nystrom_logdet", "nystrom_probes", "pcg_lanczos",
    "nystrom_dM_quadratic", "nystrom_trace_Minv_dM", "nlml_estimate_preconditioned",
    "afn_split", "fsai_pattern", "fsai_pattern_gaps", "afn_factors", "afn_matrix", "afn_apply_inverse",
    "afn_logdet", "afn_logdet_grad", "afn_dG", "afn_dM", "afn_probes", "nlml_estimate_afn",
]

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# Kernels (Sec. 2.1)
# ---------------------------------------------------------------------------

def kernel(kind: str, r: np.ndarray, ell: float) -> np.ndarray:
    """Windowed sub-kernel kappa_s as a function of the distance r = |x - y|_2.

    Sec. 2.1, eq. (2.2): Gaussian exp(-r^2 / (2 ell^2)) and Matern(1/2)
    exp(-r / ell); the Matern(3/2) kernel of the remark in Sec. 4,
    (1 + sqrt(3) r / l) exp(-sqrt(3) r / l) with l = sqrt(3) ell, i.e.
    (1 + r / ell) exp(-r / ell); and two of the further kernels named in
    Sec. 4 (generalisation), normalised to kappa(0) = 1 with c = ell: the
    inverse multiquadric (r^2 + c^2)^{-1/2} c = (1 + r^2/ell^2)^{-1/2} and
    the sinc kernel sin(r / ell) / (r / ell). None carries sigma_f (it
    multiplies the sum). A complex ``r`` evaluates the same formulas (used
    by ``kernel_taylor``)."""
    r = _as_arg(r)
    if kind == "gauss":
        return np.exp(-(r * r) / (2.0 * ell * ell))
    if kind == "matern12":
        return np.exp(-r / ell)
    if kind == "matern32":
        return (1.0 + r / ell) * np.exp(-r / ell)
    if kind == "imq":
        return 1.0 / np.sqrt(1.0 + (r / ell) ** 2)
    if kind == "sinc":
        if np.iscomplexobj(r):
            return np.sin(r / ell) / (r / ell)
        return np.sinc(r / (ell * math.pi))   # numpy's sinc(x) = sin(pi x) / (pi x)
    raise ValueError(kind)


def kernel_der_ell(kind: str, r: np.ndarray, ell: float) -> np.ndarray:
    """Derivative of kappa_s with respect to ell, Sec. 2.1 eq. (2.3):
    Gaussian r^2/ell^3 kappa^G, Matern(1/2) r/ell^2 kappa^M; Matern(3/2):
    d/dell (1 + r/ell) e^{-r/ell} = r^2/ell^3 e^{-r/ell}."""
    r = _as_arg(r)
    if kind == "gauss":
        return (r * r) / ell ** 3 * kernel(kind, r, ell)
    if kind == "matern12":
        return r / ell ** 2 * kernel(kind, r, ell)
    if kind == "matern32":
        return (r * r) / ell ** 3 * np.exp(-r / ell)
    if kind == "imq":
        # d/dell (1 + r^2/ell^2)^{-1/2} = r^2/ell^3 (1 + r^2/ell^2)^{-3/2}
        return (r * r) / ell ** 3 * (1.0 + (r / ell) ** 2) ** -1.5
    if kind == "sinc":
        # d/dell [ell sin(u) / r], u = r / ell: (sin(u)/u - cos(u)) / ell, and
        # for small u its series u^2/3 - u^4/30 + u^6/840 - u^8/45360 (the
        # closed form cancels there)
        u = r / ell
        with np.errstate(divide="ignore", invalid="ignore"):
            closed = (np.sin(u) / u - np.cos(u)) / ell
        u2 = u * u
        series = u2 * (1.0 / 3 - u2 * (1.0 / 30 - u2 * (1.0 / 840 - u2 / 45360))) / ell
        return np.where(np.abs(u) < 0.05, series, closed)
    raise ValueError(kind)


def _as_arg(r):
    r = np.asarray(r)
    return r.astype(np.complex128) if np.iscomplexobj(r) else r.astype(np.float64)


def window_points(X: np.ndarray, window) -> np.ndarray:
    """x_i^{W_s}: the columns of X listed in the window W_s (Sec. 2.1)."""
    return np.asarray(X, dtype=np.float64)[:, list(window)]


# ---------------------------------------------------------------------------
# O1: dense additive kernel sum (Sec. 2.1 eqs. (2.1)-(2.3))
# ---------------------------------------------------------------------------

def _dense_window_apply(kind, xw, V, ell, rows, der):
    n = xw.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    out = np.zeros((len(rows), V.shape[1]))
    f = kernel_der_ell if der else kernel
    step = max(1, 2_000_000 // max(n, 1))
    for a in range(0, len(rows), step):
        ri = rows[a:a + step]
        diff = xw[ri, None, :] - xw[None, :, :]
        r = np.sqrt(np.sum(diff * diff, axis=-1))
        out[a:a + step] = f(kind, r, ell) @ V
    return out


def dense_matvec(X, windows, kind, ell, sigma_f, sigma_eps, V, rows=None,
                 add_noise=True):
    """(K_hat V)[rows] with K_hat = sigma_f^2 sum_s K_s + sigma_eps^2 I.

    Sec. 2.1: the additive kernel eq. (2.1) with the windowed sub-kernels of
    eq. (2.2), regularised by sigma_eps^2 I (Sec. 1). ``rows`` selects output
    rows (every output row still sums over all n points)."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    out = 0.0
    for w in windows:
        out = out + _dense_window_apply(kind, window_points(X, w), V, ell, rows, False)
    out = sigma_f ** 2 * out
    if add_noise:
        vr = V if rows is None else V[np.asarray(rows)]
        out = out + sigma_eps ** 2 * vr
    return out


def dense_deriv_matvec(X, windows, kind, ell, sigma_f, sigma_eps, V, which,
                       rows=None):
    """(dK_hat/dtheta V)[rows] for theta in {"ell", "sigma_f", "sigma_eps"}.

    Sec. 2.1: dK_hat/dell = sigma_f^2 sum_s K_s^der (eq. (2.3));
    dK_hat/dsigma_f = 2 sigma_f sum_s K_s; dK_hat/dsigma_eps = 2 sigma_eps I."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    if which == "sigma_eps":
        vr = V if rows is None else V[np.asarray(rows)]
        return 2.0 * sigma_eps * vr
    der = which == "ell"
    out = 0.0
    for w in windows:
        out = out + _dense_window_apply(kind, window_points(X, w), V, ell, rows, der)
    if which == "ell":
        return sigma_f ** 2 * out
    if which == "sigma_f":
        return 2.0 * sigma_f * out
    raise ValueError(which)


def dense_matrix(X, windows, kind, ell, sigma_f, sigma_eps, which=None):
    """K_hat (or one of its derivative matrices) as an explicit n x n array."""
    n = X.shape[0]
    E = np.eye(n)
    if which is None:
        return dense_matvec(X, windows, kind, ell, sigma_f, sigma_eps, E)
    return dense_deriv_matvec(X, windows, kind, ell, sigma_f, sigma_eps, E, which)


# ---------------------------------------------------------------------------
# O2: Fourier-truncated sum (Sec. 3.1 eqs. (3.1)-(3.3), Sec. 3.2)
# ---------------------------------------------------------------------------

def kernel_taylor(kind: str, a: float, ell: float, p: int, der: bool = False,
                  M: int = 256) -> np.ndarray:
    """Taylor coefficients f^(j)(a) / j!, j < p, of f = kappa (or its
    ell-derivative) as a function of r, by Cauchy's integral formula
    c_j = (1 / 2 pi i) closed-integral f(z) (z - a)^{-j-1} dz on the circle
    |z - a| = a/2, discretised by the trapezoid rule with M nodes (exact up
    to aliasing c_{j+M} rho^M for a function analytic on the disc; every
    kernel here is analytic on it: the inverse multiquadric's branch points
    r = +-i ell lie outside it)."""
    rho = 0.5 * a
    theta = TWO_PI * np.arange(M) / M
    z = a + rho * np.exp(1j * theta)
    f = (kernel_der_ell if der else kernel)(kind, z, ell)
    return np.array([np.real(np.mean(f * np.exp(-1j * j * theta))) / rho ** j
                     for j in range(p)])


def boundary_polynomial(kind: str, ell: float, eps_b: float, p: int, der: bool = False):
    """Outer boundary regularisation of kappa_R (Sec. 3.1 mentions smoothing
    the outer boundary and sets it to zero; the construction is the standard
    one of the NFFT fast summation literature it cites): on the layer
    a = 1/2 - eps_b < r < 1/2 the radial kernel is replaced by the two-point
    Taylor polynomial T of degree 2p - 1 with T^(j)(a) = f^(j)(a) and, at
    r = 1/2, T = f(1/2) and T^(j) = 0 for 1 <= j < p; for r >= 1/2 kappa_R is
    the constant f(1/2), so its periodic continuation is p - 1 times
    continuously differentiable. The value f(1/2) at the outer end is a
    reading (the paper does not fix it).

    Returns e with T(r) = sum_q e_q ((r - a) / eps_b)^q, from the 2p x 2p
    linear system of the 2p conditions in the scaled variable, solved
    exactly in rational arithmetic (the system is a confluent Vandermonde
    matrix, too ill-conditioned at p = 8 for a floating-point solve)."""
    from fractions import Fraction
    a = 0.5 - eps_b
    c = kernel_taylor(kind, a, ell, p, der)
    f_half = float((kernel_der_ell if der else kernel)(kind, np.array(0.5), ell))
    n2 = 2 * p
    A = [[Fraction(0)] * n2 for _ in range(n2)]
    rhs = [Fraction(0)] * n2
    for j in range(p):
        # d^j/ds^j of s^q at s = 0 and s = 1, s = (r - a) / eps_b
        A[j][j] = Fraction(math.factorial(j))
        for q in range(j, n2):
            A[p + j][q] = Fraction(math.factorial(q) // math.factorial(q - j))
        rhs[j] = Fraction(math.factorial(j)) * Fraction(float(c[j] * eps_b ** j))
        rhs[p + j] = Fraction(f_half) if j == 0 else Fraction(0)
    # Gaussian elimination (exact, so any nonzero pivot will do)
    for col in range(n2):
        piv = next(r for r in range(col, n2) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        for r in range(col + 1, n2):
            if A[r][col] != 0:
                m = A[r][col] / A[col][col]
                A[r] = [x - m * y for x, y in zip(A[r], A[col])]
                rhs[r] -= m * rhs[col]
    e = [Fraction(0)] * n2
    for col in range(n2 - 1, -1, -1):
        acc = rhs[col] - sum(A[col][k] * e[k] for k in range(col + 1, n2))
        e[col] = acc / A[col][col]
    return np.array([float(v) for v in e])


def kernel_regularised(kind: str, r, ell: float, eps_b: float, p: int, der: bool = False):
    """kappa_R of Sec. 3.1 with outer boundary smoothing (see
    ``boundary_polynomial``): kappa for r <= 1/2 - eps_b, the boundary
    polynomial on the layer, kappa(1/2) beyond r = 1/2. With eps_b = 0 or
    p = 0 it is kappa itself."""
    r = np.asarray(r, dtype=np.float64)
    f = (kernel_der_ell if der else kernel)
    out = f(kind, r, ell)
    if eps_b <= 0 or p <= 0:
        return out
    a = 0.5 - eps_b
    e = boundary_polynomial(kind, ell, eps_b, p, der)
    layer = (r > a) & (r < 0.5)
    sl = (r[layer] - a) / eps_b
    out[layer] = sum(e[q] * sl ** q for q in range(2 * p))
    out[r >= 0.5] = float(f(kind, np.array(0.5), ell))
    return out


def index_set(N: int) -> np.ndarray:
    """I_N = {-N/2, ..., N/2 - 1} (Sec. 3.1, one dimension)."""
    if N % 2:
        raise ValueError("N must be even")
    return np.arange(-N // 2, N // 2)


def fourier_coeffs(kind: str, ell: float, N: int, d: int, der: bool = False,
                   boundary=None):
    """Discrete Fourier coefficients b_k(kappa_R), k in I_N^d.

    Sec. 3.1 eq. (3.2): b_k = N^{-d} sum_{l in I_N^d} kappa_R(l/N) e^{-2 pi i l.k/N}.
    The samples l/N lie in [-1/2, 1/2)^d, where kappa_R is kappa itself (no
    boundary smoothing, the paper's setting) or, with ``boundary = (eps_b,
    p)``, the regularised kernel of ``kernel_regularised``. With der=True the
    samples are those of the ell-derivative kernel (Sec. 3.2). The
    d-dimensional sum is evaluated one axis at a time (the exponential
    factorises over the axes).
    Returns a complex array indexed [k_1 + N/2, ..., k_d + N/2]."""
    idx = index_set(N)
    grids = np.meshgrid(*([idx / N] * d), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    eps_b, p = boundary if boundary is not None else (0.0, 0)
    samples = kernel_regularised(kind, r, ell, eps_b, p, der).astype(np.complex128)
    F = np.exp(-1j * TWO_PI * np.outer(idx, idx) / N) / N   # F[k, l]
    b = samples
    for axis in range(d):
        b = np.moveaxis(np.tensordot(F, b, axes=([1], [axis])), 0, axis)
    return b


def _exp_factors(x, N, sign):
    """Per-axis factors e^{sign 2 pi i k_t x_t}, shape (d, n, N)."""
    k = index_set(N)
    return [np.exp(sign * 1j * TWO_PI * np.outer(x[:, t], k)) for t in range(x.shape[1])]


def ndft_adjoint(x, V, N, chunk=4096):
    """c_k = sum_j v_j e^{-2 pi i k.x_j} for k in I_N^d (the inner sum of
    eq. (3.3), i.e. the exact adjoint NDFT). x: (n, d); V: (n, R).
    Returns complex (N,)*d + (R,).

    The exponential factorises over the axes, so for a chunk of points the
    sum over j is one matrix product: [prod_{t<d} e_t(j, k_t)]^T times
    [e_d(j, k_d) v_j]. Chunks of points are summed in order."""
    x = np.asarray(x, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    n, d = x.shape
    R = V.shape[1]
    out = np.zeros((N ** (d - 1), N * R), dtype=np.complex128)
    for a in range(0, n, chunk):
        E = _exp_factors(x[a:a + chunk], N, -1.0)
        m = E[0].shape[0]
        left = np.ones((m, 1), dtype=np.complex128)
        for t in range(d - 1):
            left = (left[:, :, None] * E[t][:, None, :]).reshape(m, -1)
        right = (E[d - 1][:, :, None] * V[a:a + chunk, None, :]).reshape(m, N * R)
        out += left.T @ right
    return out.reshape((N,) * d + (R,))


def ndft(x, C, N, chunk=256):
    """f(x_i) = sum_{k in I_N^d} C_k e^{2 pi i k.x_i} (the outer sum of
    eq. (3.3), i.e. the exact NDFT). C: complex (N,)*d + (R,). Returns (n, R)
    complex. The sum is taken one axis at a time (the exponential
    factorises), for a chunk of points at once."""
    x = np.asarray(x, dtype=np.float64)
    n, d = x.shape
    R = C.shape[-1]
    out = np.zeros((n, R), dtype=np.complex128)
    for a in range(0, n, chunk):
        E = _exp_factors(x[a:a + chunk], N, +1.0)
        m = E[0].shape[0]
        T = E[0] @ C.reshape(N, -1)                    # sum over k_1: (m, N^(d-1) R)
        for t in range(1, d):
            T = np.einsum("mkx,mk->mx", T.reshape(m, N, -1), E[t])
        out[a:a + chunk] = T.reshape(m, R)
    return out


def _truncated_window_apply(kind, xw, V, ell, N, der, rows, boundary=None):
    d = xw.shape[1]
    b = fourier_coeffs(kind, ell, N, d, der, boundary)
    c = ndft_adjoint(xw, V, N)
    f = b[..., None] * c
    xo = xw if rows is None else xw[np.asarray(rows)]
    return np.real(ndft(xo, f, N))


def truncated_matvec(X, windows, kind, ell, sigma_f, sigma_eps, V, N, rows=None,
                     add_noise=True, boundary=None):
    """K_hat V with every sub-kernel replaced by its truncated Fourier series.

    Sec. 3.1: per window, h(x_i) = Re sum_{k in I_N} b_k (sum_j v_j
    e^{-2 pi i k.x_j}) e^{2 pi i k.x_i} (eq. (3.3)); the approximate
    products of the windows are summed and weighted (end of Sec. 3.1):
    sigma_f^2 sum_s h_s + sigma_eps^2 v. ``N`` is an int or one per window;
    ``boundary = (eps_b, p)`` smooths kappa_R's outer boundary."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Ns = [N] * len(windows) if np.isscalar(N) else list(N)
    out = 0.0
    for w, Nw in zip(windows, Ns):
        out = out + _truncated_window_apply(kind, window_points(X, w), V, ell, Nw,
                                            False, rows, boundary)
    out = sigma_f ** 2 * out
    if add_noise:
        vr = V if rows is None else V[np.asarray(rows)]
        out = out + sigma_eps ** 2 * vr
    return out


def truncated_deriv_matvec(X, windows, kind, ell, sigma_f, sigma_eps, V, N, which,
                           rows=None, boundary=None):
    """Derivative operators of the truncated sum. For ell the coefficients are
    those of the derivative kernel, which Sec. 3.2 eq. (3.4) shows equal the
    ell-derivative of the truncated series; sigma_f and sigma_eps as in
    Sec. 2.1. With boundary smoothing the derivative kernel is regularised
    by the same construction, which is linear in the kernel's values and
    derivatives at the layer's ends, so it is the ell-derivative of the
    regularised kernel."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    if which == "sigma_eps":
        vr = V if rows is None else V[np.asarray(rows)]
        return 2.0 * sigma_eps * vr
    Ns = [N] * len(windows) if np.isscalar(N) else list(N)
    out = 0.0
    for w, Nw in zip(windows, Ns):
        out = out + _truncated_window_apply(kind, window_points(X, w), V, ell, Nw,
                                            which == "ell", rows, boundary)
    if which == "ell":
        return sigma_f ** 2 * out
    if which == "sigma_f":
        return 2.0 * sigma_f * out
    raise ValueError(which)


def truncated_operators(X, windows, kind, ell, sigma_f, sigma_eps, V, N, rows=None):
    """K_hat V and the three derivative operators applied to V, all from the
    truncated sum of Sec. 3.1 eq. (3.3): per window the inner sums
    c_k = sum_j v_j e^{-2 pi i k.x_j} are formed once and weighted by b_k of
    the kernel and of its ell-derivative (Sec. 3.2 eq. (3.4)); then
    K_hat V = sigma_f^2 sum_s h_s + sigma_eps^2 V, dK/dell V = sigma_f^2
    sum_s h_s^der, dK/dsigma_f V = 2 sigma_f sum_s h_s, dK/dsigma_eps V =
    2 sigma_eps V (Sec. 2.1). Returns a dict with keys "K", "ell", "sigma_f",
    "sigma_eps", each (len(rows) or n, R)."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Ns = [N] * len(windows) if np.isscalar(N) else list(N)
    h = 0.0
    hd = 0.0
    for w, Nw in zip(windows, Ns):
        xw = window_points(X, w)
        d = xw.shape[1]
        c = ndft_adjoint(xw, V, Nw)
        xo = xw if rows is None else xw[np.asarray(rows)]
        b = fourier_coeffs(kind, ell, Nw, d, False)
        bd = fourier_coeffs(kind, ell, Nw, d, True)
        h = h + np.real(ndft(xo, b[..., None] * c, Nw))
        hd = hd + np.real(ndft(xo, bd[..., None] * c, Nw))
    vr = V if rows is None else V[np.asarray(rows)]
    return {"K": sigma_f ** 2 * h + sigma_eps ** 2 * vr, "ell": sigma_f ** 2 * hd,
            "sigma_f": 2.0 * sigma_f * h, "sigma_eps": 2.0 * sigma_eps * vr}


def truncated_forms(X, windows, kind, ell, sigma_f, sigma_eps, G, V, N):
    """sum_r G_r^T Op V_r for Op = K_hat and its three derivative operators,
    with the truncated sum of Sec. 3.1 eq. (3.3) summed against G:
    G^T K_s V = sum_i G_i Re sum_k b_k c_k(V) e^{2 pi i k.x_i}
              = Re sum_k b_k c_k(V) conj(c_k(G))   (G real),
    c_k(.) the inner sums; b_k of the ell-derivative kernel for "ell"
    (Sec. 3.2 eq. (3.4)). Returns a dict with keys "K", "ell", "sigma_f",
    "sigma_eps" (floats)."""
    G = np.asarray(G, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if G.ndim == 1:
        G = G[:, None]
    if V.ndim == 1:
        V = V[:, None]
    Ns = [N] * len(windows) if np.isscalar(N) else list(N)
    q = 0.0
    qd = 0.0
    for w, Nw in zip(windows, Ns):
        xw = window_points(X, w)
        d = xw.shape[1]
        cv = ndft_adjoint(xw, V, Nw)
        cg = ndft_adjoint(xw, G, Nw)
        prod = (np.conj(cg) * cv).sum(axis=-1)
        q += float(np.real(np.sum(fourier_coeffs(kind, ell, Nw, d, False) * prod)))
        qd += float(np.real(np.sum(fourier_coeffs(kind, ell, Nw, d, True) * prod)))
    gv = float(np.sum(G * V))
    return {"K": sigma_f ** 2 * q + sigma_eps ** 2 * gv, "ell": sigma_f ** 2 * qd,
            "sigma_f": 2.0 * sigma_f * q, "sigma_eps": 2.0 * sigma_eps * gv}


# ---------------------------------------------------------------------------
# NFFT (Appendix A): Kaiser-Bessel window, adjoint NFFT and NFFT
# ---------------------------------------------------------------------------

def bins(x: np.ndarray, n_os: int) -> np.ndarray:
    """Index of the oversampled-grid cell that holds each coordinate:
    floor(x * n_os). The grid points are l / n_os (Appendix A)."""
    return np.floor(np.asarray(x, dtype=np.float64) * n_os).astype(np.int64)


def kb_shape(sigma_os: float) -> float:
    """Kaiser-Bessel shape parameter b = pi (2 - 1/sigma) (Appendix A)."""
    return math.pi * (2.0 - 1.0 / sigma_os)


def kb_window(x, n_os: int, s: int, sigma_os: float = 2.0):
    """Truncated Kaiser-Bessel window phi(x) of Appendix A:
    (1/pi) sinh(b sqrt(s^2 - n_os^2 x^2)) / sqrt(s^2 - n_os^2 x^2) for
    |x| <= s / n_os, and 0 outside (the truncation). At the support edge the
    value is the limit b/pi."""
    b = kb_shape(sigma_os)
    x = np.asarray(x, dtype=np.float64)
    t = s * s - (n_os * x) ** 2
    out = np.zeros_like(x)
    inside = t >= 0
    root = np.sqrt(np.where(inside, t, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        val = np.where(root > 0, np.sinh(b * root) / np.where(root > 0, root, 1.0), b)
    out[inside] = val[inside] / math.pi
    return out


def kb_window_hat(k, n_os: int, s: int, sigma_os: float = 2.0):
    """Fourier transform of the Kaiser-Bessel window at frequency k:
    (1/n_os) I0(s sqrt(b^2 - (2 pi k / n_os)^2)). This is the standard
    closed form (Kaiser-Bessel transform pair) that Appendix A refers to; it
    holds for |2 pi k / n_os| < b, which every k in I_N satisfies."""
    b = kb_shape(sigma_os)
    w = TWO_PI * np.asarray(k, dtype=np.float64) / n_os
    if np.any(np.abs(w) >= b):
        raise ValueError("frequency outside the I0 branch")
    return scipy.special.i0(s * np.sqrt(b * b - w * w)) / n_os


def _spread_grid(x, V, n_os, s, sigma_os):
    """G_l = sum_j v_j prod_t phi~(x_jt - l_t/n_os), l in I_{n_os}^d, stored
    at array index l + n_os/2 (l taken modulo n_os: phi~ is the 1-periodic
    window)."""
    n, d = x.shape
    R = V.shape[1]
    G = np.zeros((n_os,) * d + (R,))
    base = np.floor(x * n_os).astype(np.int64) - s          # (n, d)
    offs = np.arange(0, 2 * s + 1)            # every l with |x n_os - l| <= s
    # per-axis weights w[t][j, o] = phi(x_jt - (base_jt + o)/n_os)
    W = [kb_window(x[:, t, None] - (base[:, t, None] + offs[None, :]) / n_os,
                   n_os, s, sigma_os) for t in range(d)]
    for o in np.ndindex(*([len(offs)] * d)):
        w = np.ones(n)
        idx = []
        for t in range(d):
            w = w * W[t][:, o[t]]
            idx.append((base[:, t] + offs[o[t]] + n_os // 2) % n_os)
        np.add.at(G, tuple(idx), w[:, None] * V)
    return G


def _interp_grid(x, G, n_os, s, sigma_os):
    """f_i = sum_l G_l prod_t phi~(x_it - l_t/n_os) (sparse window sum,
    Appendix A step 3)."""
    n, d = x.shape
    out = np.zeros((n,) + G.shape[d:], dtype=G.dtype)
    base = np.floor(x * n_os).astype(np.int64) - s
    offs = np.arange(0, 2 * s + 1)
    W = [kb_window(x[:, t, None] - (base[:, t, None] + offs[None, :]) / n_os,
                   n_os, s, sigma_os) for t in range(d)]
    for o in np.ndindex(*([len(offs)] * d)):
        w = np.ones(n)
        idx = []
        for t in range(d):
            w = w * W[t][:, o[t]]
            idx.append((base[:, t] + offs[o[t]] + n_os // 2) % n_os)
        out += w[:, None] * G[tuple(idx)]
    return out


def _window_hat_nd(N, n_os, s, sigma_os, d):
    """prod_t phi_hat(k_t) on I_N^d."""
    h = kb_window_hat(index_set(N), n_os, s, sigma_os)
    out = h
    for _ in range(d - 1):
        out = np.multiply.outer(out, h)
    return out


def nfft_adjoint(x, V, N, s, sigma_os=2.0):
    """Approximate c_k = sum_j v_j e^{-2 pi i k.x_j}, k in I_N^d, by the adjoint
    of the three NFFT steps of Appendix A: spread onto the oversampled grid
    with the periodised window, FFT, divide by the window's Fourier transform
    and by n_os^d."""
    x = np.asarray(x, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    d = x.shape[1]
    n_os = int(round(sigma_os * N))
    G = _spread_grid(x, V, n_os, s, sigma_os)
    # sum_l G_l e^{-2 pi i k.l/n_os} with l centred: move l=0 to index 0
    Gh = np.fft.fftn(np.fft.ifftshift(G, axes=tuple(range(d))), axes=tuple(range(d)))
    sel = np.ix_(*([index_set(N) % n_os] * d))
    Gk = Gh[sel]
    return Gk / (n_os ** d * _window_hat_nd(N, n_os, s, sigma_os, d))[..., None]


def nfft(x, C, N, s, sigma_os=2.0):
    """Approximate f(x_i) = sum_k C_k e^{2 pi i k.x_i} by the three NFFT steps of
    Appendix A: (1) divide by the window's Fourier transform and zero-pad to
    I_{n_os}; (2) FFT to grid values g_l (with the 1/n_os^d of the inverse
    transform); (3) sparse window sum at the points."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    n_os = int(round(sigma_os * N))
    Gk = np.zeros((n_os,) * d + C.shape[d:], dtype=np.complex128)
    sel = np.ix_(*([index_set(N) % n_os] * d))
    Gk[sel] = C / _window_hat_nd(N, n_os, s, sigma_os, d)[..., None]
    g = np.fft.ifftn(Gk, axes=tuple(range(d)))            # includes 1/n_os^d
    g = np.fft.fftshift(g, axes=tuple(range(d)))            # index l + n_os/2
    return _interp_grid(x, g, n_os, s, sigma_os)


def nfft_fastsum_matvec(X, windows, kind, ell, sigma_f, sigma_eps, V, N, s,
                        sigma_os=2.0, add_noise=True, boundary=None):
    """The method itself on the CPU: eq. (3.3) with the inner sum by the
    adjoint NFFT and the outer sum by the NFFT (Sec. 3.1 and Appendix A),
    real part, then the weighted window sum."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    Ns = [N] * len(windows) if np.isscalar(N) else list(N)
    out = 0.0
    for w, Nw in zip(windows, Ns):
        xw = window_points(X, w)
        b = fourier_coeffs(kind, ell, Nw, xw.shape[1], boundary=boundary)
        chat = nfft_adjoint(xw, V, Nw, s, sigma_os)
        out = out + np.real(nfft(xw, b[..., None] * chat, Nw, s, sigma_os))
    out = sigma_f ** 2 * out
    if add_noise:
        out = out + sigma_eps ** 2 * V
    return out


# ---------------------------------------------------------------------------
# Iterative solvers and the likelihood (Sec. 1)
# ---------------------------------------------------------------------------

# Lanczos breakdown floor of the NLML estimators (FP64): a CG-Lanczos column
# whose relative residual has fallen to this level has reached an invariant
# Krylov subspace to working precision, so its Lanczos matrix ends there (the
# Gauss quadrature of e_1^T f(T) e_1 is then exact to that level; further
# steps would divide rounding-level residual norms by each other).
LANCZOS_BREAKDOWN = 1e-12


def cg(apply_A, B, rtol=1e-4, maxit=200, fixed_iters=None, breakdown=0.0):
    """Conjugate gradients for A X = B, one independent recursion per column,
    zero initial guess, stopping when |b - A x|_2 / |b|_2 <= rtol (Sec. 1 and
    the CG setup of Sec. 5.1). With ``fixed_iters`` every column runs that
    many steps (the Lanczos use), or stops earlier once its relative residual
    is <= ``breakdown``. Returns X, iterations, relative residuals, and the
    per-column alpha and beta sequences."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, R = B.shape
    X = np.zeros_like(B)
    iters = np.zeros(R, dtype=np.int64)
    relres = np.ones(R)
    alphas = [[] for _ in range(R)]
    betas = [[] for _ in range(R)]
    for c in range(R):
        b = B[:, c]
        bn = np.linalg.norm(b)
        if bn == 0:
            relres[c] = 0.0
            continue
        x = np.zeros(n)
        r = b.copy()
        p = r.copy()
        rr = r @ r
        lim = fixed_iters if fixed_iters is not None else maxit
        for it in range(lim):
            q = apply_A(p[:, None])[:, 0]
            a = rr / (p @ q)
            x = x + a * p
            r = r - a * q
            rr_new = r @ r
            beta = rr_new / rr
            alphas[c].append(a)
            betas[c].append(beta)
            iters[c] = it + 1
            relres[c] = math.sqrt(rr_new) / bn
            rr = rr_new
            if fixed_iters is None and relres[c] <= rtol:
                break
            if fixed_iters is not None and relres[c] <= breakdown:
                break
            p = r + beta * p
        X[:, c] = x
    return X, iters, relres, alphas, betas


def pcg(apply_A, apply_Minv, B, rtol=1e-4, maxit=200):
    """Preconditioned conjugate gradients for A X = B, one recursion per
    column, zero initial guess, stopping on the unpreconditioned relative
    residual |b - A x|_2 / |b|_2 <= rtol (Sec. 1, Sec. 5.1). Returns X,
    iterations, relative residuals."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, R = B.shape
    X = np.zeros_like(B)
    iters = np.zeros(R, dtype=np.int64)
    relres = np.ones(R)
    for c in range(R):
        b = B[:, c]
        bn = np.linalg.norm(b)
        if bn == 0:
            relres[c] = 0.0
            continue
        x = np.zeros(n)
        r = b.copy()
        z = apply_Minv(r[:, None])[:, 0]
        p = z.copy()
        rz = r @ z
        for it in range(maxit):
            q = apply_A(p[:, None])[:, 0]
            a = rz / (p @ q)
            x = x + a * p
            r = r - a * q
            iters[c] = it + 1
            relres[c] = np.linalg.norm(r) / bn
            if relres[c] <= rtol:
                break
            z = apply_Minv(r[:, None])[:, 0]
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        X[:, c] = x
    return X, iters, relres


def farthest_point_sampling(x, k):
    """Greedy farthest point sampling of k indices of the rows of x (Sec. 2.3,
    the landmark choice of the additive AFN preconditioner): start at index 0,
    then repeatedly take the point whose distance to the chosen set is
    largest, the lowest index among equal distances. Distances are squared
    Euclidean distances in FP64."""
    return [i for i, _, _ in farthest_point_gaps(x, k)]


def farthest_point_gaps(x, k):
    """``farthest_point_sampling(x, k)`` with, for each step, the chosen
    index, its distance to the set chosen before it and the gap between that
    distance and the largest distance of any other point (inf for the first
    point). A gap near zero marks a near-tie, where a distance evaluated with
    other rounding may decide differently."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    k = min(k, n)
    out = [(0, np.inf, np.inf)]
    dist = np.full(n, np.inf)
    for _ in range(1, k):
        last = x[out[-1][0]]
        dist = np.minimum(dist, np.sum((x - last) ** 2, axis=1))
        i = int(np.argmax(dist))                # argmax returns the first maximum
        rest = np.delete(dist, i)
        out.append((i, float(dist[i]), float(dist[i] - rest.max()) if rest.size else np.inf))
    return out


def additive_landmarks(X, windows, k_total):
    """Landmarks of every feature window (ceil(k_total / P) each by farthest
    point sampling on that window's features), merged into one sorted set
    without repeats (Sec. 2.3)."""
    P = len(windows)
    kw = max(1, -(-k_total // P))
    s = set()
    for w in windows:
        s.update(farthest_point_sampling(window_points(X, w), kw))
    return sorted(s)


def landmark_jitter(B, KLL0, sigma_f, P, sigma_eps):
    """delta added to the diagonal of K_LL (not in the paper): 1e-6 sigma_f^2 P
    (1e-6 of the kernel's diagonal value), grown 100-fold, at most four
    times, while the Cholesky factorisation of G = sigma_eps^2 (K_LL + delta I)
    + B^T B fails in FP64 -- when more landmarks are requested than the
    kernel's numerical rank the landmark columns B are numerically dependent.
    KLL0 = B[L] without jitter. It is held fixed when M is differentiated."""
    BtB = np.asarray(B, dtype=np.float64).T @ np.asarray(B, dtype=np.float64)
    k = KLL0.shape[0]
    delta = 1e-6 * sigma_f ** 2 * P
    for _ in range(5):
        try:
            np.linalg.cholesky(sigma_eps ** 2 * (KLL0 + delta * np.eye(k)) + BtB)
            return delta
        except np.linalg.LinAlgError:
            delta *= 100.0
    raise np.linalg.LinAlgError("G is not positive definite for any jitter tried")


def nystrom_preconditioner(X, windows, kind, ell, sigma_f, sigma_eps, landmarks, jitter=None):
    """M = K_{:,L} (K_LL + delta I)^{-1} K_{L,:} + sigma_eps^2 I with K =
    sigma_f^2 sum_s K_s (the exact kernel of Sec. 2.1), the landmark set L and
    delta = landmark_jitter unless given -- the (1,1)-block Nystrom part of the
    additive AFN preconditioner (Sec. 2.3). Formed as a dense n x n matrix;
    returns a function applying M^{-1}."""
    n = X.shape[0]
    L = list(landmarks)
    KnL = dense_matvec(X, windows, kind, ell, sigma_f, 0.0, np.eye(n)[:, L], add_noise=False)
    delta = (landmark_jitter(KnL, KnL[L, :], sigma_f, len(windows), sigma_eps)
             if jitter is None else jitter)
    KLL = KnL[L, :] + delta * np.eye(len(L))
    M = KnL @ np.linalg.solve(KLL, KnL.T) + sigma_eps ** 2 * np.eye(n)
    M = 0.5 * (M + M.T)
    return lambda P: np.linalg.solve(M, P)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Outputs 0 .. count-1 of the SplitMix64 generator (Steele, Lea and
    Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
    started from state ``seed``: output i mixes the state seed + (i + 1) g,
    g = 0x9E3779B97F4A7C15, by z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
    z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31 (mod 2^64). Output i
    depends only on (seed, i): the generator is counter-based."""
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def rademacher_probes(n: int, R: int, seed: int) -> np.ndarray:
    """n x R Rademacher probes (Hutchinson's estimator, Sec. 1): entry (i, c)
    is +1 when the top bit of SplitMix64 output i R + c is 0, else -1."""
    z = splitmix64(seed, n * R)
    return np.where((z >> np.uint64(63)) == 0, 1.0, -1.0).reshape(n, R)


def lanczos_tridiag_from_cg(alphas, betas):
    """Lanczos tridiagonal matrix T from the CG coefficients (the standard
    CG-Lanczos relation used by stochastic Lanczos quadrature, cited in
    Sec. 1): T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    T_{j,j+1} = sqrt(beta_j)/alpha_j."""
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]
    return T


def slq_quadratic(T, znorm2):
    """Gauss quadrature estimate of z^T logm(A) z from the Lanczos matrix T of
    the Krylov space started at z: |z|^2 sum_k tau_k^2 log theta_k with
    (theta_k, u_k) the eigenpairs of T and tau_k = u_k[0] (Sec. 1, SLQ)."""
    theta, U = np.linalg.eigh(T)
    return znorm2 * float(np.sum(U[0, :] ** 2 * np.log(theta)))


def nlml_exact(K_hat, y):
    """Z = 1/2 (y^T K_hat^{-1} y + log det K_hat + n log 2 pi), Sec. 1 eq. (1.2),
    by a dense Cholesky factorisation."""
    L = np.linalg.cholesky(K_hat)
    a = np.linalg.solve(L.T, np.linalg.solve(L, y))
    n = len(y)
    return 0.5 * (y @ a + 2.0 * np.sum(np.log(np.diag(L))) + n * math.log(TWO_PI))


def nlml_estimate(apply_K, apply_dK, y, Z, lanczos_steps, rtol=1e-10, maxit=None,
                  breakdown=LANCZOS_BREAKDOWN):
    """Estimate of the NLML and its gradient with M = I (no preconditioner).

    Sec. 1 eq. (1.4) with M = I: Z~ = 1/2 (y^T alpha + (1/n_z) sum_i z_i^T
    logm(K_hat) z_i + n log 2 pi), each quadratic form by SLQ with
    ``lanczos_steps`` CG steps started at z_i. Eq. (1.5) with M = I:
    dZ~/dtheta = 1/2 (-alpha^T dK alpha + (1/n_z) sum_i u_i^T dK z_i),
    u_i = K_hat^{-1} z_i (the CG solution after ``lanczos_steps`` steps).
    alpha solves K_hat alpha = y by CG to ``rtol``.

    apply_dK: dict theta -> callable. Returns (nlml, {theta: grad})."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    n = y.shape[0]
    alpha, _, _, _, _ = cg(apply_K, y[:, None], rtol=rtol,
                           maxit=maxit if maxit is not None else 10 * n)
    alpha = alpha[:, 0]
    U, _, _, al, be = cg(apply_K, Z, fixed_iters=lanczos_steps, breakdown=breakdown)
    nz = Z.shape[1]
    logdet = 0.0
    for i in range(nz):
        T = lanczos_tridiag_from_cg(al[i], be[i])
        logdet += slq_quadratic(T, float(Z[:, i] @ Z[:, i]))
    logdet /= nz
    nlml = 0.5 * (y @ alpha + logdet + n * math.log(TWO_PI))
    grads = {}
    for th, f in apply_dK.items():
        da = f(alpha[:, None])[:, 0]
        dz = f(Z)
        tr = float(np.sum(U * dz)) / nz
        grads[th] = 0.5 * (-(alpha @ da) + tr)
    return nlml, grads


# ---------------------------------------------------------------------------
# Preconditioned NLML estimate with the landmark (Nystrom) preconditioner
# (Sec. 1 eqs. (1.3)-(1.5); M from the (1,1) block of Sec. 2.3)
# ---------------------------------------------------------------------------

def nystrom_blocks(X, windows, kind, ell, sigma_f, landmarks, which=None, jitter=None,
                   sigma_eps=None):
    """B = K_{:,L}, the columns of sigma_f^2 sum_s K_s (exact kernel, Sec. 2.1)
    at the landmarks L, and K_LL = B[L, :] + delta I (delta = landmark_jitter,
    which needs sigma_eps, unless given). With which = "ell" or "sigma_f" the
    derivative of B with respect to that hyperparameter and its landmark rows
    (sigma_eps does not enter B; delta is held fixed)."""
    n = X.shape[0]
    L = list(landmarks)
    E = np.zeros((n, len(L)))
    E[L, np.arange(len(L))] = 1.0
    if which is not None:
        dB = dense_deriv_matvec(X, windows, kind, ell, sigma_f, 0.0, E, which)
        return dB, dB[L, :]
    B = dense_matvec(X, windows, kind, ell, sigma_f, 0.0, E, add_noise=False)
    delta = (landmark_jitter(B, B[L, :], sigma_f, len(windows), sigma_eps)
             if jitter is None else jitter)
    return B, B[L, :] + delta * np.eye(len(L))


def nystrom_matrix(B, KLL, s2):
    """M = B K_LL^{-1} B^T + s2 I as an explicit n x n array."""
    M = B @ np.linalg.solve(KLL, B.T) + s2 * np.eye(B.shape[0])
    return 0.5 * (M + M.T)


def nystrom_logdet(B, KLL, s2):
    """log det M for M = B K_LL^{-1} B^T + s2 I by the matrix determinant
    lemma: (n - k) log s2 + log det(s2 K_LL + B^T B) - log det K_LL."""
    n, k = B.shape
    _, ld_g = np.linalg.slogdet(s2 * KLL + B.T @ B)
    _, ld_k = np.linalg.slogdet(KLL)
    return (n - k) * math.log(s2) + ld_g - ld_k


def nystrom_probes(B, KLL, sigma_eps, Wn, Wk):
    """Probes with covariance M: z_i = sigma_eps Wn[:, i] + B C^{-T} Wk[:, i],
    C the lower Cholesky factor of K_LL, for given vectors w_i = [Wn; Wk][:, i]
    (n + k entries, E[w w^T] = I): cov(z) = sigma_eps^2 I + B K_LL^{-1} B^T."""
    C = np.linalg.cholesky(KLL)
    T = np.linalg.solve(C.T, np.asarray(Wk, dtype=np.float64))
    return sigma_eps * np.asarray(Wn, dtype=np.float64) + B @ T


def pcg_lanczos(apply_A, apply_Minv, B, steps, breakdown=0.0):
    """PCG with zero initial guess and ``steps`` steps per column (fewer if
    the relative residual |r|_2 / |b|_2 falls to ``breakdown``), recording
    the alpha and beta sequences (which give the Lanczos matrix of
    M^{-1/2} A M^{-1/2} started at M^{-1/2} b, by the same CG-Lanczos relation
    as in lanczos_tridiag_from_cg) and r_0^T M^{-1} r_0 = b^T M^{-1} b.
    Returns X, alphas, betas, rz0."""
    B = np.asarray(B, dtype=np.float64)
    n, R = B.shape
    X = np.zeros_like(B)
    alphas, betas, rz0 = [[] for _ in range(R)], [[] for _ in range(R)], np.zeros(R)
    for c in range(R):
        x = np.zeros(n)
        r = B[:, c].copy()
        z = apply_Minv(r[:, None])[:, 0]
        p = z.copy()
        rz = r @ z
        rz0[c] = rz
        bn = np.linalg.norm(B[:, c])
        for _ in range(steps):
            q = apply_A(p[:, None])[:, 0]
            a = rz / (p @ q)
            x = x + a * p
            r = r - a * q
            z = apply_Minv(r[:, None])[:, 0]
            rz_new = r @ z
            b = rz_new / rz
            alphas[c].append(a)
            betas[c].append(b)
            if np.linalg.norm(r) <= breakdown * bn:
                break
            p = z + b * p
            rz = rz_new
        X[:, c] = x
    return X, alphas, betas, rz0


def nystrom_dM_quadratic(B, KLL, dB, dKLL, P):
    """p_i^T (dM/dtheta) p_i for the columns p_i of P, theta in {ell,
    sigma_f}: dM = dB K^{-1} B^T + B K^{-1} dB^T - B K^{-1} dK_LL K^{-1} B^T
    (K = K_LL), so p^T dM p = 2 a^T K^{-1} e - a^T K^{-1} dK_LL K^{-1} a with
    a = B^T p, e = dB^T p."""
    A = B.T @ P
    Ed = dB.T @ P
    KiA = np.linalg.solve(KLL, A)
    return 2.0 * np.sum(KiA * Ed, axis=0) - np.sum(KiA * (dKLL @ KiA), axis=0)


def nystrom_trace_Minv_dM(B, KLL, dB, dKLL, s2):
    """tr(M^{-1} dM/dtheta) for theta in {ell, sigma_f} (dense: the oracle)."""
    M = nystrom_matrix(B, KLL, s2)
    dM = dB @ np.linalg.solve(KLL, B.T)
    dM = dM + dM.T - B @ np.linalg.solve(KLL, dKLL) @ np.linalg.solve(KLL, B.T)
    return float(np.trace(np.linalg.solve(M, dM)))


def nlml_estimate_preconditioned(apply_K, apply_dK, y, Wn, Wk, lanczos_steps, B, KLL, dB,
                                 landmarks, sigma_eps, rtol=1e-10, maxit=None,
                                 breakdown=LANCZOS_BREAKDOWN):
    """Estimate of the NLML and its gradient with the landmark preconditioner
    M = B K_LL^{-1} B^T + sigma_eps^2 I (Sec. 2.3).

    Sec. 1 eq. (1.4): Z~ = 1/2 (y^T alpha + log det M + (1/n_z) sum_i q_i +
    n log 2 pi), log det M exact (eq. (1.3)), q_i the SLQ estimate of
    z~_i^T logm(M^{-1/2} K_hat M^{-1/2}) z~_i from ``lanczos_steps`` PCG steps on
    K_hat x = z_i, with z~_i = M^{-1/2} z_i (|z~_i|^2 = z_i^T M^{-1} z_i). The
    probes z_i = sigma_eps wn_i + B C^{-T} wk_i have covariance M, so the z~_i
    have covariance I and the mean of the q_i estimates tr(Delta log).

    Eq. (1.5): dZ~/dtheta = 1/2 (-alpha^T dK alpha + tr(M^{-1} dM) + (1/n_z)
    sum_i s_i), s_i = u_i^T dK p_i - p_i^T dM p_i with u_i = K_hat^{-1} z_i
    (the PCG iterate) and p_i = M^{-1} z_i: for cov(z) = M its mean is
    tr(K_hat^{-1} dK) - tr(M^{-1} dM), the trace of (M^{-1}K_hat)^{-1}
    d(M^{-1} K_hat). dB: {"ell": dB/dell, "sigma_f": dB/dsigma_f} (from
    nystrom_blocks), landmarks: the rows L of B; for sigma_eps, dM = 2 sigma_eps I.
    alpha solves K_hat alpha = y by PCG to ``rtol``. Returns (nlml, {theta: grad})."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    n = y.shape[0]
    s2 = sigma_eps ** 2
    M = nystrom_matrix(B, KLL, s2)

    def Minv(P):
        return np.linalg.solve(M, P)

    alpha, _, _ = pcg(apply_K, Minv, y[:, None], rtol=rtol,
                      maxit=maxit if maxit is not None else 10 * n)
    alpha = alpha[:, 0]
    Z = nystrom_probes(B, KLL, sigma_eps, Wn, Wk)
    U, al, be, rz0 = pcg_lanczos(apply_K, Minv, Z, lanczos_steps, breakdown=breakdown)
    nz = Z.shape[1]
    quad = 0.0
    for i in range(nz):
        quad += slq_quadratic(lanczos_tridiag_from_cg(al[i], be[i]), float(rz0[i]))
    logdet = nystrom_logdet(B, KLL, s2) + quad / nz
    nlml = 0.5 * (y @ alpha + logdet + n * math.log(TWO_PI))
    P = Minv(Z)
    L = list(landmarks)
    grads = {}
    for th, f in apply_dK.items():
        da = f(alpha[:, None])[:, 0]
        dz = f(P)
        if th == "sigma_eps":
            tr_m = 2.0 * sigma_eps * float(np.trace(np.linalg.inv(M)))
            pdp = 2.0 * sigma_eps * np.sum(P * P, axis=0)
        else:
            dKLL = dB[th][L]
            tr_m = nystrom_trace_Minv_dM(B, KLL, dB[th], dKLL, s2)
            pdp = nystrom_dM_quadratic(B, KLL, dB[th], dKLL, P)
        s = np.sum(U * dz, axis=0) - pdp
        grads[th] = 0.5 * (-(alpha @ da) + tr_m + float(np.mean(s)))
    return nlml, grads



# ---------------------------------------------------------------------------
# Additive AFN preconditioner (Sec. 2.3): Cholesky of the landmark block and
# a factorised sparse approximate inverse (FSAI) of the Schur complement
# ---------------------------------------------------------------------------

def afn_split(n, landmarks):
    """(L, F): the landmark indices (ascending) and the remaining indices
    (ascending) -- the 2 x 2 block structure of the AFN preconditioner."""
    L = sorted(set(int(i) for i in landmarks))
    mask = np.ones(n, dtype=bool)
    mask[L] = False
    return L, [int(i) for i in np.nonzero(mask)[0]]


def fsai_pattern(X, windows, landmarks, fill, rows=None):
    """Sparsity pattern of the lower-triangular FSAI factor of the Schur
    complement (Sec. 2.3: 'fill level'). Rows and columns are the positions
    t = 0 .. |F|-1 of the non-landmark points F in ascending index order.
    Row t holds t and its min(fill - 1, t) nearest earlier positions u < t,
    by the squared Euclidean distance over the window features (every
    window's features in window order) in FP64; ties go to the lower
    position. Returns one ascending position list per row (t last), for
    every row or for the positions listed in ``rows``."""
    return [J for J, _ in fsai_pattern_gaps(X, windows, landmarks, fill, rows)]


def fsai_pattern_gaps(X, windows, landmarks, fill, rows=None):
    """``fsai_pattern`` with, per row, the gap between the fill-th and the
    (fill-1)-th smallest distance (inf when every earlier position is
    kept): a gap near zero marks a near-tie, where a distance evaluated with
    other rounding may decide differently. Returns (J_t, gap_t) pairs."""
    n = X.shape[0]
    _, F = afn_split(n, landmarks)
    cols = [c for w in windows for c in w]
    x = np.asarray(X, dtype=np.float64)[F][:, cols]
    out = []
    for t in (range(len(F)) if rows is None else rows):
        if t == 0 or fill <= 1:
            out.append(([t], np.inf))
            continue
        acc = np.zeros(t)
        for c in range(len(cols)):
            acc = acc + (x[:t, c] - x[t, c]) ** 2
        order = np.lexsort((np.arange(t), acc))     # by distance, then position
        gap = float(acc[order[fill - 1]] - acc[order[fill - 2]]) if t > fill - 1 else np.inf
        out.append((sorted(int(u) for u in order[:fill - 1]) + [t], gap))
    return out


def afn_factors(X, windows, kind, ell, sigma_f, sigma_eps, landmarks, fill):
    """The factors of the AFN preconditioner for K_hat = sigma_f^2 sum_s K_s +
    sigma_eps^2 I (exact kernel, Sec. 2.1). With the landmarks L first and
    the rest F after them,

        K_hat = [K_LL  K_LF]   S = K_FF - K_FL K_LL^{-1} K_LF (Schur complement)
                [K_FL  K_FF],

    (all blocks of K_hat, noise included). Row t of the FSAI factor G is
    g / sqrt(g_t), g solving S[J_t, J_t] g = e_t on the pattern J_t of
    fsai_pattern, so that G S G^T has unit diagonal and G^T G approximates
    S^{-1}. Returns (L, F, K_LL, K_FL, S, G, J) as dense arrays."""
    n = X.shape[0]
    L, F = afn_split(n, landmarks)
    K = dense_matrix(X, windows, kind, ell, sigma_f, sigma_eps)
    KLL = K[np.ix_(L, L)]
    KFL = K[np.ix_(F, L)]
    S = K[np.ix_(F, F)] - KFL @ np.linalg.solve(KLL, KFL.T)
    S = 0.5 * (S + S.T)
    J = fsai_pattern(X, windows, landmarks, fill)
    G = np.zeros((len(F), len(F)))
    for t, Jt in enumerate(J):
        e = np.zeros(len(Jt))
        e[-1] = 1.0
        g = np.linalg.solve(S[np.ix_(Jt, Jt)], e)
        G[t, Jt] = g / math.sqrt(g[-1])
    return L, F, KLL, KFL, S, G, J


def afn_matrix(L, F, KLL, KFL, G):
    """M = Phi diag(K_LL, (G^T G)^{-1}) Phi^T, Phi = [I 0; K_FL K_LL^{-1} I],
    as an explicit n x n array in the original point order."""
    n = len(L) + len(F)
    k = len(L)
    Phi = np.eye(n)
    Phi[k:, :k] = np.linalg.solve(KLL, KFL.T).T
    D = np.zeros((n, n))
    D[:k, :k] = KLL
    D[k:, k:] = np.linalg.inv(G.T @ G)
    Mp = Phi @ D @ Phi.T
    order = list(L) + list(F)
    M = np.zeros((n, n))
    M[np.ix_(order, order)] = 0.5 * (Mp + Mp.T)
    return M


def afn_apply_inverse(L, F, KLL, KFL, G, V):
    """M^{-1} V in the three block steps of the factorised form:
    t = V_F - K_FL K_LL^{-1} V_L; w = G^T G t;
    out_L = K_LL^{-1} (V_L - K_FL^T w), out_F = w."""
    V = np.asarray(V, dtype=np.float64)
    VL, VF = V[L], V[F]
    y = np.linalg.solve(KLL, VL)
    t = VF - KFL @ y
    w = G.T @ (G @ t)
    out = np.zeros_like(V)
    out[F] = w
    out[L] = np.linalg.solve(KLL, VL - KFL.T @ w)
    return out


def afn_logdet(KLL, G):
    """log det M = log det K_LL - 2 sum_t log G_tt (block triangular factors)."""
    _, ld = np.linalg.slogdet(KLL)
    return ld - 2.0 * float(np.sum(np.log(np.diag(G))))


def afn_logdet_grad(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, G, J, which):
    """d log det M / dtheta with the landmarks and the pattern held fixed:
    tr(K_LL^{-1} dK_LL) + sum_t G_t^T dS[J_t, J_t] G_t, because
    d log G_tt = -1/2 G_t^T dS[J_t, J_t] G_t for G_tt^2 = e_t^T S_JJ^{-1} e_t,
    and dS = dK_FF - dK_FL A - A^T dK_LF + A^T dK_LL A with A = K_LL^{-1} K_LF."""
    dK = dense_matrix(X, windows, kind, ell, sigma_f, sigma_eps, which=which)
    dLL = dK[np.ix_(L, L)]
    dFL = dK[np.ix_(F, L)]
    A = np.linalg.solve(KLL, KFL.T)
    dS = dK[np.ix_(F, F)] - dFL @ A - A.T @ dFL.T + A.T @ dLL @ A
    out = float(np.trace(np.linalg.solve(KLL, dLL)))
    for t, Jt in enumerate(J):
        g = G[t, Jt]
        out += float(g @ dS[np.ix_(Jt, Jt)] @ g)
    return out


def _afn_dblocks(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, which):
    """dK_LL, dK_FL and dS (derivatives of the blocks of K_hat and of the
    Schur complement S with respect to ``which``)."""
    dK = dense_matrix(X, windows, kind, ell, sigma_f, sigma_eps, which=which)
    dLL = dK[np.ix_(L, L)]
    dFL = dK[np.ix_(F, L)]
    A = np.linalg.solve(KLL, KFL.T)
    dS = dK[np.ix_(F, F)] - dFL @ A - A.T @ dFL.T + A.T @ dLL @ A
    return dLL, dFL, 0.5 * (dS + dS.T)


def afn_dG(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, S, G, J, which):
    """dG/dtheta with the landmarks and the pattern held fixed. Row t,
    g = G[t, J_t]: differentiating S_JJ u = e_t and g = u / sqrt(u_t) gives
    dg = -S_JJ^{-1} dS_JJ g + g (g^T dS_JJ g) / 2."""
    _, _, dS = _afn_dblocks(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, which)
    dG = np.zeros_like(G)
    for t, Jt in enumerate(J):
        g = G[t, Jt]
        v = dS[np.ix_(Jt, Jt)] @ g
        dG[t, Jt] = -np.linalg.solve(S[np.ix_(Jt, Jt)], v) + 0.5 * g * float(g @ v)
    return dG


def afn_dM(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, S, G, J, which):
    """dM/dtheta (dense, original point order) for M = Phi D Phi^T with
    Phi = [I 0; Xm I], Xm = K_FL K_LL^{-1}, D = diag(K_LL, (G^T G)^{-1}):
    dXm = (dK_FL - Xm dK_LL) K_LL^{-1},
    d(G^T G)^{-1} = -(G^T G)^{-1} (dG^T G + G^T dG) (G^T G)^{-1}."""
    dLL, dFL, _ = _afn_dblocks(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, which)
    dG = afn_dG(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, S, G, J, which)
    n, k = len(L) + len(F), len(L)
    Xm = np.linalg.solve(KLL, KFL.T).T
    dXm = np.linalg.solve(KLL, (dFL - Xm @ dLL).T).T
    Phi = np.eye(n)
    Phi[k:, :k] = Xm
    dPhi = np.zeros((n, n))
    dPhi[k:, :k] = dXm
    St = np.linalg.inv(G.T @ G)
    D = np.zeros((n, n))
    D[:k, :k] = KLL
    D[k:, k:] = St
    dD = np.zeros((n, n))
    dD[:k, :k] = dLL
    dD[k:, k:] = -St @ (dG.T @ G + G.T @ dG) @ St
    dMp = dPhi @ D @ Phi.T + Phi @ dD @ Phi.T + Phi @ D @ dPhi.T
    order = list(L) + list(F)
    dM = np.zeros((n, n))
    dM[np.ix_(order, order)] = 0.5 * (dMp + dMp.T)
    return dM


def afn_probes(L, F, KLL, KFL, G, Wn):
    """Probes with covariance M: z = Phi [C w_L; G^{-1} w_F] (C C^T = K_LL),
    i.e. z_L = C w_L and z_F = K_FL K_LL^{-1} z_L + G^{-1} w_F, for given
    vectors w (the columns of Wn, rows in the original point order)."""
    Wn = np.asarray(Wn, dtype=np.float64)
    C = np.linalg.cholesky(KLL)
    Z = np.zeros_like(Wn)
    zL = C @ Wn[L]
    Z[L] = zL
    Z[F] = KFL @ np.linalg.solve(KLL, zL) + np.linalg.solve(G, Wn[F])
    return Z


def nlml_estimate_afn(apply_K, apply_dK, y, Wn, lanczos_steps, X, windows, kind, ell, sigma_f,
                      sigma_eps, landmarks, fill, rtol=1e-10, maxit=None,
                      breakdown=LANCZOS_BREAKDOWN):
    """Estimate of the NLML and its gradient (Sec. 1 eqs. (1.3)-(1.5)) with the
    additive AFN preconditioner M of afn_factors (Sec. 2.3): the same
    estimator as nlml_estimate_preconditioned, with log det M = log det K_LL -
    2 sum log G_tt, tr(M^{-1} dM) = d log det M / dtheta (afn_logdet_grad),
    probes z_i = afn_probes(w_i) and p^T dM p from afn_dM. Returns (nlml,
    {theta: grad})."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    n = y.shape[0]
    L, F, KLL, KFL, S, G, J = afn_factors(X, windows, kind, ell, sigma_f, sigma_eps,
                                          landmarks, fill)

    def Minv(P):
        return afn_apply_inverse(L, F, KLL, KFL, G, P)

    alpha, _, _ = pcg(apply_K, Minv, y[:, None], rtol=rtol,
                      maxit=maxit if maxit is not None else 10 * n)
    alpha = alpha[:, 0]
    Z = afn_probes(L, F, KLL, KFL, G, Wn)
    U, al, be, rz0 = pcg_lanczos(apply_K, Minv, Z, lanczos_steps, breakdown=breakdown)
    nz = Z.shape[1]
    quad = 0.0
    for i in range(nz):
        quad += slq_quadratic(lanczos_tridiag_from_cg(al[i], be[i]), float(rz0[i]))
    logdet = afn_logdet(KLL, G) + quad / nz
    nlml = 0.5 * (y @ alpha + logdet + n * math.log(TWO_PI))
    P = Minv(Z)
    grads = {}
    for th, f in apply_dK.items():
        da = f(alpha[:, None])[:, 0]
        dz = f(P)
        tr_m = afn_logdet_grad(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, G, J, th)
        dM = afn_dM(X, windows, kind, ell, sigma_f, sigma_eps, L, F, KLL, KFL, S, G, J, th)
        s = np.sum(U * dz, axis=0) - np.sum(P * (dM @ P), axis=0)
        grads[th] = 0.5 * (-(alpha @ da) + tr_m + float(np.mean(s)))
    return nlml, grads
