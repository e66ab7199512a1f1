"""Pins of the oracle's outer boundary smoothing of kappa_R (Sec. 3.1: the
periodic extension may be smoothed at its outer boundary; the paper keeps
that smoothing at zero, this library offers it as an option).

Each check compares with something other than the oracle itself: sympy's
symbolic derivatives, scipy's Hermite (Krogh) interpolation through the same
conditions, the trigonometric interpolation property of the truncated series
on lattice points, and the dense kernel sum that the smoothed series must
approach faster than the unsmoothed one."""
import math

import numpy as np
import pytest
from scipy.interpolate import KroghInterpolator

from oracle import agp_oracle as O

KINDS = ["gauss", "matern12", "matern32", "imq", "sinc"]


def _sympy_kernel(kind, ell, der):
    sp = pytest.importorskip("sympy")
    r, l = sp.symbols("r l", positive=True)
    f = {
        "gauss": sp.exp(-r ** 2 / (2 * l ** 2)),
        "matern12": sp.exp(-r / l),
        "matern32": (1 + r / l) * sp.exp(-r / l),
        "imq": 1 / sp.sqrt(1 + r ** 2 / l ** 2),
        "sinc": sp.sin(r / l) / (r / l),
    }[kind]
    if der:
        f = sp.diff(f, l)
    return sp, r, f.subs(l, sp.Rational(str(ell)) if isinstance(ell, str) else ell)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("der", [False, True])
@pytest.mark.parametrize("ell,a", [(0.3, 0.4375), (0.08, 0.375), (1.5, 0.40625)])
def test_kernel_taylor_matches_symbolic_derivatives(kind, der, ell, a):
    sp, r, f = _sympy_kernel(kind, ell, der)
    p = 7
    c = O.kernel_taylor(kind, a, ell, p, der)
    for j in range(p):
        exact = float(sp.diff(f, r, j).subs(r, a)) / math.factorial(j)
        # absolute scale of the j-th coefficient on the circle of radius a/2
        scale = max(abs(float(f.subs(r, a))), 1e-3) / (0.5 * a) ** j
        assert abs(c[j] - exact) <= 1e-11 * scale + 1e-12 * abs(exact), (j, c[j], exact)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("der", [False, True])
@pytest.mark.parametrize("eps_b,p", [(0.125, 4), (0.0625, 3), (0.1875, 6)])
def test_boundary_polynomial_is_the_hermite_interpolant(kind, der, eps_b, p):
    """On the layer the regularised kernel is the unique polynomial of degree
    2p - 1 through p conditions at each end: scipy's Krogh interpolation
    with repeated nodes builds it from the same data independently."""
    sp, r, f = _sympy_kernel(kind, 0.3, der)
    a = 0.5 - eps_b
    ya = [float(sp.diff(f, r, j).subs(r, a)) for j in range(p)]
    yb = [float(f.subs(r, sp.Rational(1, 2)))] + [0.0] * (p - 1)
    krogh = KroghInterpolator([a] * p + [0.5] * p, ya + yb)
    rr = np.linspace(a, 0.5, 41)[1:-1]
    got = O.kernel_regularised(kind, rr, 0.3, eps_b, p, der)
    want = krogh(rr)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("kind", KINDS)
def test_regularised_kernel_inside_and_outside(kind):
    eps_b, p = 0.125, 4
    r = np.linspace(0.0, 0.375, 50)
    np.testing.assert_array_equal(O.kernel_regularised(kind, r, 0.3, eps_b, p),
                                  O.kernel(kind, r, 0.3))
    far = np.array([0.5, 0.6, 0.8660254])
    np.testing.assert_allclose(O.kernel_regularised(kind, far, 0.3, eps_b, p),
                               O.kernel(kind, np.array(0.5), 0.3), rtol=0, atol=0)
    # no smoothing requested: the plain kernel everywhere
    r = np.linspace(0.0, 0.86, 30)
    np.testing.assert_array_equal(O.kernel_regularised(kind, r, 0.3, 0.0, 4),
                                  O.kernel(kind, r, 0.3))
    np.testing.assert_array_equal(O.kernel_regularised(kind, r, 0.3, 0.125, 0),
                                  O.kernel(kind, r, 0.3))


@pytest.mark.parametrize("kind", ["gauss", "matern32", "sinc"])
def test_regularised_kernel_smooth_across_both_ends(kind):
    """kappa_R is p - 1 times continuously differentiable at r = a and at
    r = 1/2: one-sided finite-difference derivatives (orders 0..2) agree."""
    eps_b, p, ell = 0.125, 4, 0.3
    a = 0.5 - eps_b
    h = 1e-5

    def one_sided(r0, side, order):
        pts = r0 + side * h * np.arange(1, 5)   # four points on one side
        vals = O.kernel_regularised(kind, pts, ell, eps_b, p)
        # fit a cubic through the samples and differentiate it at r0
        coef = np.polyfit(pts - r0, vals, 3)
        return np.polyval(np.polyder(coef, order), 0.0) if order else np.polyval(coef, 0.0)

    for r0 in (a, 0.5):
        # errors of the one-sided cubic fit: O(h^(4 - order)) plus rounding
        for order, tol in ((0, 1e-10), (1, 1e-6), (2, 1e-3)):
            left, right = one_sided(r0, -1, order), one_sided(r0, +1, order)
            scale = max(1.0, abs(left))
            assert abs(left - right) <= tol * scale, (r0, order, left, right)


def _ball_points(n, d, radius, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x * radius * rng.uniform(0, 1, (n, 1)) ** (1.0 / d)


def test_smoothed_series_interpolates_on_lattice_points():
    """The truncated series interpolates kappa_R at every lattice difference;
    points of the lattice inside the ball of radius 1/4 - eps_b/2 have
    differences where kappa_R = kappa, so the smoothed truncated sum equals
    the dense sum there to rounding."""
    N, eps_b, p = 16, 0.125, 4
    rng = np.random.default_rng(3)
    grid = np.stack(np.meshgrid(*([O.index_set(N) / N] * 2), indexing="ij"), -1).reshape(-1, 2)
    inside = grid[np.linalg.norm(grid, axis=1) <= 0.25 - eps_b / 2]
    X = inside[rng.permutation(len(inside))[:30]]
    V = rng.standard_normal((len(X), 2))
    for kind in ("gauss", "matern12", "sinc"):
        dense = O.dense_matvec(X, [[0, 1]], kind, 0.2, 1.0, 0.0, V)
        tr = O.truncated_matvec(X, [[0, 1]], kind, 0.2, 1.0, 0.0, V, N,
                                boundary=(eps_b, p))
        np.testing.assert_allclose(tr, dense, rtol=0, atol=1e-12 * np.abs(dense).max())


@pytest.mark.parametrize("kind,ell", [("gauss", 0.3), ("matern32", 0.3)])
def test_smoothing_shrinks_the_truncation_error(kind, ell):
    """With a smooth periodic kappa_R the Fourier coefficients decay faster,
    so the truncated sum comes closer to the dense sum (measured on points
    in the ball where both describe the same kernel)."""
    d, N, eps_b, p = 3, 32, 0.125, 4
    X = _ball_points(250, d, 0.25 - eps_b / 2, seed=1)
    V = np.random.default_rng(2).standard_normal((len(X), 1))
    dense = O.dense_matvec(X, [[0, 1, 2]], kind, ell, 1.0, 0.0, V)
    plain = O.truncated_matvec(X, [[0, 1, 2]], kind, ell, 1.0, 0.0, V, N)
    smooth = O.truncated_matvec(X, [[0, 1, 2]], kind, ell, 1.0, 0.0, V, N,
                                boundary=(eps_b, p))
    e_plain = np.linalg.norm(plain - dense) / np.linalg.norm(dense)
    e_smooth = np.linalg.norm(smooth - dense) / np.linalg.norm(dense)
    # measured: 1.7e-3 -> 1.9e-4 (Gaussian), 1.5e-3 -> 1.5e-4 (Matern(3/2))
    assert e_smooth < e_plain / 5, (e_plain, e_smooth)


@pytest.mark.parametrize("kind", ["gauss", "matern32", "imq"])
def test_derivative_consistency_with_smoothing(kind):
    """Eq. (3.4) with kappa_R smoothed: the truncated sum of the regularised
    derivative kernel equals the ell-derivative of the regularised truncated
    sum (central differences, O(h^2))."""
    d, N, eps_b, p, ell, h = 2, 16, 0.125, 4, 0.25, 1e-4
    X = _ball_points(60, d, 0.25 - eps_b / 2, seed=4)
    V = np.random.default_rng(5).standard_normal((len(X), 2))
    b = (eps_b, p)
    fp = O.truncated_matvec(X, [[0, 1]], kind, ell + h, 1.0, 0.0, V, N, boundary=b)
    fm = O.truncated_matvec(X, [[0, 1]], kind, ell - h, 1.0, 0.0, V, N, boundary=b)
    fd = (fp - fm) / (2 * h)
    an = O.truncated_deriv_matvec(X, [[0, 1]], kind, ell, 1.0, 0.0, V, N, "ell", boundary=b)
    np.testing.assert_allclose(an, fd, rtol=0, atol=1e-6 * np.abs(an).max())


def test_nfft_fastsum_with_smoothing_matches_truncated_sum():
    """The method on the CPU (adjoint NFFT, multiply, NFFT; Appendix A) with
    the smoothed coefficients reproduces the smoothed truncated sum to the
    Kaiser-Bessel window error (s = 5, sigma = 2)."""
    d, N, eps_b, p = 2, 16, 0.125, 4
    X = _ball_points(400, d, 0.25 - eps_b / 2, seed=6)
    V = np.random.default_rng(7).standard_normal((len(X), 2))
    b = (eps_b, p)
    fast = O.nfft_fastsum_matvec(X, [[0, 1]], "gauss", 0.2, 1.0, 0.1, V, N, 5, boundary=b)
    trunc = O.truncated_matvec(X, [[0, 1]], "gauss", 0.2, 1.0, 0.1, V, N, boundary=b)
    assert np.linalg.norm(fast - trunc) / np.linalg.norm(trunc) < 1e-8
    plain = O.truncated_matvec(X, [[0, 1]], "gauss", 0.2, 1.0, 0.1, V, N)
    assert np.linalg.norm(plain - trunc) / np.linalg.norm(trunc) > 1e-6   # smoothing changed it
