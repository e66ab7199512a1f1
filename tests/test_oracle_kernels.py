"""Pins of the oracle's dense additive kernel sum (Sec. 2.1) to values that do
not come from the oracle itself: textbook constants, closed forms of special
configurations, invariances and a brute-force loop on tiny inputs."""
import math

import numpy as np
import pytest

import oracle as O

KINDS = ["gauss", "matern12", "matern32", "imq", "sinc"]


def test_kernel_textbook_values():
    # exp(-1/2) and exp(-1): the kernels at distance r = ell.
    assert O.kernel("gauss", 0.7, 0.7) == pytest.approx(0.6065306597126334, rel=1e-15)
    assert O.kernel("matern12", 0.7, 0.7) == pytest.approx(0.36787944117144233, rel=1e-15)
    assert O.kernel("gauss", 0.0, 0.3) == 1.0
    assert O.kernel("matern12", 0.0, 0.3) == 1.0


@pytest.mark.parametrize("kind", KINDS)
def test_kernel_der_is_ell_derivative(kind):
    # eq. (2.3) against a central difference of eq. (2.2) in ell.
    r = np.linspace(0.0, 0.9, 37)
    ell, h = 0.31, 1e-5
    fd = (O.kernel(kind, r, ell + h) - O.kernel(kind, r, ell - h)) / (2 * h)
    np.testing.assert_allclose(O.kernel_der_ell(kind, r, ell), fd, rtol=1e-8, atol=1e-10)


def _brute(X, windows, kind, ell, sf, se, v):
    n = len(X)
    out = [0.0] * n
    for i in range(n):
        acc = 0.0
        for w in windows:
            for j in range(n):
                d2 = 0.0
                for f in w:
                    d2 += (X[i][f] - X[j][f]) ** 2
                r = math.sqrt(d2)
                if kind == "gauss":
                    k = math.exp(-d2 / (2 * ell * ell))
                elif kind == "matern12":
                    k = math.exp(-r / ell)
                elif kind == "matern32":   # the form of Sec. 4 with l = sqrt(3) ell
                    l = math.sqrt(3.0) * ell
                    k = (1 + math.sqrt(3.0) * r / l) * math.exp(-math.sqrt(3.0) * r / l)
                elif kind == "imq":        # c (r^2 + c^2)^{-1/2}, c = ell
                    k = ell / math.sqrt(d2 + ell * ell)
                else:                      # sinc: sin(r / ell) / (r / ell)
                    k = 1.0 if r == 0 else math.sin(r / ell) * ell / r
                acc += k * v[j]
        out[i] = sf * sf * acc + se * se * v[i]
    return np.array(out)


@pytest.mark.parametrize("kind", KINDS)
def test_dense_matches_brute_force_loop(kind):
    rng = np.random.default_rng(5)
    X = rng.uniform(-0.24, 0.24, size=(7, 5))
    v = rng.standard_normal(7)
    windows = [[0, 2], [1, 3, 4]]
    got = O.dense_matvec(X, windows, kind, 0.2, 1.3, 0.4, v)[:, 0]
    want = _brute(X.tolist(), windows, kind, 0.2, 1.3, 0.4, v.tolist())
    np.testing.assert_allclose(got, want, rtol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_dense_identical_points_closed_form(kind):
    # All points equal: every K_s is the all-ones matrix, so
    # K_hat v = sigma_f^2 P (sum v) 1 + sigma_eps^2 v.
    X = np.full((9, 6), 0.11)
    v = np.arange(9, dtype=float) - 3.0
    windows = [[0, 1, 2], [3, 4], [5]]
    got = O.dense_matvec(X, windows, kind, 0.3, 0.8, 0.5, v)[:, 0]
    want = 0.8 ** 2 * 3 * v.sum() + 0.25 * v
    np.testing.assert_allclose(got, want, rtol=1e-14)


def test_dense_two_points_closed_form():
    # Two points 0.1 apart in feature 1 only; window {0,1}: off-diagonal
    # entry exp(-0.01 / (2*0.04)) = exp(-0.125).
    X = np.array([[0.0, 0.0, 0.2], [0.0, 0.1, -0.2]])
    K = O.dense_matrix(X, [[0, 1]], "gauss", 0.2, 1.0, 0.0)
    np.testing.assert_allclose(K, [[1.0, 0.8824969025845955], [0.8824969025845955, 1.0]],
                               rtol=1e-15)


@pytest.mark.parametrize("kind", KINDS)
def test_dense_translation_invariance_and_unused_features(kind):
    rng = np.random.default_rng(6)
    X = rng.uniform(-0.2, 0.2, size=(40, 6))
    v = rng.standard_normal((40, 2))
    windows = [[0, 1, 2], [4, 5]]
    a = O.dense_matvec(X, windows, kind, 0.25, 1.0, 0.1, v)
    Y = X + np.array([0.03, -0.02, 0.01, 0.0, 0.04, -0.01])
    Y[:, 3] = rng.uniform(-0.2, 0.2, size=40)       # feature 3 is in no window
    b = O.dense_matvec(Y, windows, kind, 0.25, 1.0, 0.1, v)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13)


def test_gaussian_window_is_product_of_one_dimensional_kernels():
    rng = np.random.default_rng(7)
    X = rng.uniform(-0.24, 0.24, size=(30, 3))
    K012 = O.dense_matrix(X, [[0, 1, 2]], "gauss", 0.15, 1.0, 0.0)
    K0 = O.dense_matrix(X, [[0]], "gauss", 0.15, 1.0, 0.0)
    K1 = O.dense_matrix(X, [[1]], "gauss", 0.15, 1.0, 0.0)
    K2 = O.dense_matrix(X, [[2]], "gauss", 0.15, 1.0, 0.0)
    np.testing.assert_allclose(K012, K0 * K1 * K2, rtol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_dense_symmetric_positive_definite(kind):
    rng = np.random.default_rng(8)
    X = rng.uniform(-0.24, 0.24, size=(50, 5))
    K = O.dense_matrix(X, [[0, 1], [2, 3, 4]], kind, 0.2, 1.0, 0.05)
    np.testing.assert_array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("which", ["ell", "sigma_f", "sigma_eps"])
def test_dense_derivative_operators_match_finite_differences(kind, which):
    rng = np.random.default_rng(9)
    X = rng.uniform(-0.24, 0.24, size=(25, 4))
    v = rng.standard_normal((25, 2))
    W = [[0, 1], [2, 3]]
    th = {"ell": 0.21, "sigma_f": 0.9, "sigma_eps": 0.3}
    h = 1e-4

    def f(dt):
        t = dict(th)
        t[which] += dt
        return O.dense_matvec(X, W, kind, t["ell"], t["sigma_f"], t["sigma_eps"], v)

    # fourth-order central difference
    fd = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)
    got = O.dense_deriv_matvec(X, W, kind, th["ell"], th["sigma_f"], th["sigma_eps"], v, which)
    np.testing.assert_allclose(got, fd, rtol=1e-8, atol=1e-9 * np.abs(got).max())


def test_dense_rows_subset():
    rng = np.random.default_rng(10)
    X = rng.uniform(-0.24, 0.24, size=(60, 3))
    v = rng.standard_normal((60, 3))
    full = O.dense_matvec(X, [[0, 1, 2]], "gauss", 0.2, 1.0, 0.1, v)
    rows = [0, 17, 59]
    np.testing.assert_allclose(O.dense_matvec(X, [[0, 1, 2]], "gauss", 0.2, 1.0, 0.1, v,
                                              rows=rows), full[rows], rtol=1e-14)


def test_matern32_textbook_values():
    # (1 + sqrt(3) r / l) exp(-sqrt(3) r / l) with l = sqrt(3) ell (the remark
    # of Sec. 4): at r = ell this is 2 / e.
    assert O.kernel("matern32", 0.4, 0.4) == pytest.approx(2.0 / math.e, rel=1e-15)
    assert O.kernel("matern32", 0.0, 0.3) == 1.0
    l = math.sqrt(3.0) * 0.25
    r = 0.6
    assert O.kernel("matern32", r, 0.25) == pytest.approx(
        (1 + math.sqrt(3.0) * r / l) * math.exp(-math.sqrt(3.0) * r / l), rel=1e-14)


def test_imq_and_sinc_textbook_values():
    # inverse multiquadric at r = ell: 1/sqrt(2); at r = sqrt(3) ell: 1/2
    assert O.kernel("imq", 0.3, 0.3) == pytest.approx(1.0 / math.sqrt(2.0), rel=1e-15)
    assert O.kernel("imq", math.sqrt(3.0) * 0.2, 0.2) == pytest.approx(0.5, rel=1e-15)
    # sinc: zero at r = pi ell, 2/pi at r = pi ell / 2, 1 at r = 0
    assert abs(O.kernel("sinc", math.pi * 0.1, 0.1)) < 1e-15
    assert O.kernel("sinc", math.pi * 0.05, 0.1) == pytest.approx(2.0 / math.pi, rel=1e-15)
    assert O.kernel("sinc", 0.0, 0.1) == 1.0


def test_sinc_derivative_series_meets_closed_form():
    # the small-argument series and the closed form agree where both are
    # accurate, and the derivative vanishes at r = 0
    ell = 0.2
    r = np.array([0.04, 0.049, 0.0501, 0.06]) * ell
    u = r / ell
    closed = (np.sin(u) / u - np.cos(u)) / ell
    np.testing.assert_allclose(O.kernel_der_ell("sinc", r, ell), closed, rtol=1e-11)
    assert O.kernel_der_ell("sinc", 0.0, ell) == 0.0
