"""Pins of the oracle's Fourier coefficients b_k (Sec. 3.1 eq. (3.2)) and of
the truncated sum (eq. (3.3)) to the paper's worked example, closed forms and
properties that hold by the mathematics."""
import cmath
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = ["gauss", "matern12", "matern32", "imq", "sinc"]


def _read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            rows.append((int(k), float(v)))
    return rows


def test_worked_example_matern_1d():
    # Sec. 3.1, figure of the 1-D kernel approximation: Matern(1/2),
    # ell = 0.3, m = N = 8, coefficients printed to 16 digits.
    b = O.fourier_coeffs("matern12", 0.3, 8, 1)
    for k, val in _read_golden("worked_example_matern12_1d.txt"):
        assert b[k + 4].real == pytest.approx(val, rel=2e-15, abs=1e-17)
        assert abs(b[k + 4].imag) < 1e-16


@pytest.mark.parametrize("N,ell", [(8, 0.3), (16, 0.07), (32, 0.5), (64, 0.2)])
def test_matern_1d_geometric_series_closed_form(N, ell):
    # b_k = (1/N) sum_{l=-N/2}^{N/2-1} q^{|l|} e^{-2 pi i l k/N}, q = e^{-1/(N ell)}:
    # 1 + 2 Re[z (1 - z^{N/2-1}) / (1 - z)] + q^{N/2} (-1)^k with z = q e^{i theta}.
    b = O.fourier_coeffs("matern12", ell, N, 1)
    q = math.exp(-1.0 / (N * ell))
    for k in range(-N // 2, N // 2):
        z = q * cmath.exp(2j * math.pi * k / N)
        M = N // 2 - 1
        geo = z * (1 - z ** M) / (1 - z)
        want = (1.0 + 2.0 * geo.real + q ** (N // 2) * (-1) ** k) / N
        assert b[k + N // 2].real == pytest.approx(want, rel=1e-12, abs=1e-16)


def _gauss_hat_1d(w, ell):
    # Fourier transform of exp(-x^2 / (2 ell^2)) (e^{-2 pi i w x} convention).
    return math.sqrt(2 * math.pi) * ell * np.exp(-2 * math.pi ** 2 * ell ** 2 * w ** 2)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_gaussian_coeffs_equal_aliased_fourier_transform(d):
    # Small ell: the periodisation error exp(-1/(8 ell^2)) is ~1e-22 and
    # b_k = sum_m kappa_hat(k + m N) (aliasing formula, Sec. 4.1).
    N, ell = 32, 0.05
    b = O.fourier_coeffs("gauss", ell, N, d)
    k = O.index_set(N)
    h1 = sum(_gauss_hat_1d(k + m * N, ell) for m in range(-3, 4))
    want = h1
    for _ in range(d - 1):
        want = np.multiply.outer(want, h1)
    np.testing.assert_allclose(b.real, want, rtol=1e-12, atol=1e-15 * want.max())
    assert np.max(np.abs(b.imag)) < 1e-16


def test_gaussian_coeffs_separable():
    b3 = O.fourier_coeffs("gauss", 0.27, 16, 3)
    b1 = O.fourier_coeffs("gauss", 0.27, 16, 1)
    np.testing.assert_allclose(b3, np.multiply.outer(np.multiply.outer(b1, b1), b1),
                               rtol=1e-12, atol=1e-17)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [1, 2, 3])
def test_coeffs_real_even(kind, d):
    N = 16
    b = O.fourier_coeffs(kind, 0.2, N, d)
    assert np.max(np.abs(b.imag)) < 1e-15
    # b_{-k} = b_k where both lie in I_N (index k -> N - k for k != -N/2)
    inner = tuple(slice(1, None) for _ in range(d))
    bi = b.real[inner]
    np.testing.assert_allclose(bi, np.flip(bi), rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [1, 2, 3])
def test_derivative_coeffs_equal_ell_derivative(kind, d):
    # Sec. 3.2 eq. (3.4): the coefficients of the derivative kernel are the
    # ell-derivative of the coefficients.
    N, ell, h = 16, 0.23, 1e-4
    f = lambda e: O.fourier_coeffs(kind, e, N, d)
    # fourth-order central difference
    fd = (8 * (f(ell + h) - f(ell - h)) - (f(ell + 2 * h) - f(ell - 2 * h))) / (12 * h)
    np.testing.assert_allclose(O.fourier_coeffs(kind, ell, N, d, der=True), fd,
                               rtol=1e-8, atol=1e-11)


def _lattice_points(rng, n, p, N):
    # points on the lattice (1/N) Z^p inside [-1/4, 1/4)^p
    return rng.integers(-N // 4, N // 4, size=(n, p)) / N


@pytest.mark.parametrize("kind", KINDS)
def test_truncated_equals_dense_on_lattice(kind):
    # kappa_RF interpolates kappa at the N-periodic lattice (Sec. 3.1 figure
    # caption), and every difference of lattice points in [-1/4, 1/4) is a
    # lattice point of [-1/2, 1/2). So on lattice points the truncated sum IS
    # the dense sum, for any kernel and any d.
    rng = np.random.default_rng(11)
    N = 16
    X = _lattice_points(rng, 80, 6, N)
    v = rng.standard_normal((80, 3))
    W = [[0, 1, 2], [3, 4], [5]]
    t = O.truncated_matvec(X, W, kind, 0.17, 1.1, 0.3, v, N)
    dns = O.dense_matvec(X, W, kind, 0.17, 1.1, 0.3, v)
    np.testing.assert_allclose(t, dns, rtol=1e-11, atol=1e-12)
    for which in ["ell", "sigma_f", "sigma_eps"]:
        t = O.truncated_deriv_matvec(X, W, kind, 0.17, 1.1, 0.3, v, N, which)
        dns = O.dense_deriv_matvec(X, W, kind, 0.17, 1.1, 0.3, v, which)
        np.testing.assert_allclose(t, dns, rtol=1e-10, atol=1e-11)


def test_truncated_converges_to_dense_small_ell():
    rng = np.random.default_rng(12)
    X = rng.uniform(-0.24, 0.24, size=(300, 3))
    v = rng.standard_normal((300, 2))
    W = [[0, 1], [2]]
    t = O.truncated_matvec(X, W, "gauss", 0.03, 1.0, 0.0, v, 64)
    dns = O.dense_matvec(X, W, "gauss", 0.03, 1.0, 0.0, v)
    assert np.linalg.norm(t - dns) / np.linalg.norm(dns) < 1e-7


@pytest.mark.parametrize("kind", KINDS)
def test_truncated_symmetric(kind):
    # With the real part taken, w^T K_RF v = v^T K_RF w to rounding.
    rng = np.random.default_rng(13)
    X = rng.uniform(-0.24, 0.24, size=(120, 5))
    v = rng.standard_normal((120, 1))
    w = rng.standard_normal((120, 1))
    W = [[0, 1, 2], [3, 4]]
    a = float(w[:, 0] @ O.truncated_matvec(X, W, kind, 0.3, 1.0, 0.2, v, 16)[:, 0])
    b = float(v[:, 0] @ O.truncated_matvec(X, W, kind, 0.3, 1.0, 0.2, w, 16)[:, 0])
    assert a == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("kind", KINDS)
def test_truncated_derivative_operator_matches_fd(kind):
    rng = np.random.default_rng(14)
    X = rng.uniform(-0.24, 0.24, size=(90, 5))
    v = rng.standard_normal((90, 2))
    W = [[0, 1, 2], [3, 4]]
    h = 1e-4
    f = lambda e: O.truncated_matvec(X, W, kind, e, 1.2, 0.1, v, 16)
    fd = (8 * (f(0.25 + h) - f(0.25 - h)) - (f(0.25 + 2 * h) - f(0.25 - 2 * h))) / (12 * h)
    got = O.truncated_deriv_matvec(X, W, kind, 0.25, 1.2, 0.1, v, 16, "ell")
    np.testing.assert_allclose(got, fd, rtol=1e-8, atol=1e-9 * np.abs(got).max())


def test_truncated_rows_and_window_bandwidths():
    rng = np.random.default_rng(15)
    X = rng.uniform(-0.24, 0.24, size=(70, 5))
    v = rng.standard_normal((70, 2))
    W = [[0, 1, 2], [3, 4]]
    full = O.truncated_matvec(X, W, "gauss", 0.3, 1.0, 0.1, v, [8, 16])
    rows = [3, 40, 69]
    np.testing.assert_allclose(
        O.truncated_matvec(X, W, "gauss", 0.3, 1.0, 0.1, v, [8, 16], rows=rows),
        full[rows], rtol=1e-13)
    one = (O.truncated_matvec(X, [W[0]], "gauss", 0.3, 1.0, 0.0, v, 8)
           + O.truncated_matvec(X, [W[1]], "gauss", 0.3, 1.0, 0.0, v, 16) + 0.01 * v)
    np.testing.assert_allclose(full, one, rtol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_truncated_operators_pinned(kind):
    # all four operators from one set of inner sums: on lattice points they
    # are the dense operators (the interpolation property above), and off the
    # lattice the ell and sigma_f operators are the central differences of the
    # K output in those parameters (sigma_eps: of the noise term)
    rng = np.random.default_rng(16)
    N = 16
    X = _lattice_points(rng, 60, 5, N)
    v = rng.standard_normal((60, 2))
    W = [[0, 1, 2], [3, 4]]
    ops = O.truncated_operators(X, W, kind, 0.2, 1.3, 0.4, v, N)
    np.testing.assert_allclose(ops["K"], O.dense_matvec(X, W, kind, 0.2, 1.3, 0.4, v),
                               rtol=1e-11, atol=1e-12)
    for which in ["ell", "sigma_f", "sigma_eps"]:
        np.testing.assert_allclose(
            ops[which], O.dense_deriv_matvec(X, W, kind, 0.2, 1.3, 0.4, v, which),
            rtol=1e-10, atol=1e-11)
    Xr = rng.uniform(-0.24, 0.24, size=(50, 5))
    rows = [0, 7, 49]
    ops = O.truncated_operators(Xr, W, kind, 0.25, 1.2, 0.3, v[:50], [8, 16], rows=rows)
    h = 1e-5
    th = {"ell": 0.25, "sigma_f": 1.2, "sigma_eps": 0.3}
    for which in th:
        up, dn = dict(th), dict(th)
        up[which] += h
        dn[which] -= h
        fu = O.truncated_operators(Xr, W, kind, up["ell"], up["sigma_f"], up["sigma_eps"],
                                   v[:50], [8, 16], rows=rows)["K"]
        fd = O.truncated_operators(Xr, W, kind, dn["ell"], dn["sigma_f"], dn["sigma_eps"],
                                   v[:50], [8, 16], rows=rows)["K"]
        np.testing.assert_allclose(ops[which], (fu - fd) / (2 * h), rtol=1e-6,
                                   atol=1e-7 * np.abs(ops[which]).max())


@pytest.mark.parametrize("kind", KINDS)
def test_truncated_forms_pinned(kind):
    # on lattice points the forms are those of the dense operators; off the
    # lattice they are the column sums of G * (operator V) and symmetric in
    # (G, V)
    rng = np.random.default_rng(17)
    N = 16
    X = _lattice_points(rng, 50, 5, N)
    G = rng.standard_normal((50, 3))
    V = rng.standard_normal((50, 3))
    W = [[0, 1, 2], [3, 4]]
    f = O.truncated_forms(X, W, kind, 0.2, 1.3, 0.4, G, V, N)
    assert f["K"] == pytest.approx(float(np.sum(G * O.dense_matvec(X, W, kind, 0.2, 1.3, 0.4, V))),
                                   rel=1e-10)
    for which in ["ell", "sigma_f", "sigma_eps"]:
        ref = float(np.sum(G * O.dense_deriv_matvec(X, W, kind, 0.2, 1.3, 0.4, V, which)))
        assert f[which] == pytest.approx(ref, rel=1e-9, abs=1e-11), which
    Xr = rng.uniform(-0.24, 0.24, size=(50, 5))
    f = O.truncated_forms(Xr, W, kind, 0.25, 1.2, 0.3, G, V, [8, 16])
    ops = O.truncated_operators(Xr, W, kind, 0.25, 1.2, 0.3, V, [8, 16])
    g = O.truncated_forms(Xr, W, kind, 0.25, 1.2, 0.3, V, G, [8, 16])
    for which in ops:
        assert f[which] == pytest.approx(float(np.sum(G * ops[which])), rel=1e-11), which
        assert f[which] == pytest.approx(g[which], rel=1e-11), which


def test_ndft_pair_single_point():
    # c_k of a single unit mass at x is e^{-2 pi i k.x}; the NDFT of
    # C_k = delta_{k,k0} is e^{2 pi i k0.x}.
    x = np.array([[0.1, -0.2]])
    c = O.ndft_adjoint(x, np.ones((1, 1)), 8)
    assert c[3 + 4, -2 + 4, 0] == pytest.approx(cmath.exp(-2j * math.pi * (3 * 0.1 - 2 * -0.2)))
    C = np.zeros((8, 8, 1), complex)
    C[1 + 4, -4 + 4, 0] = 1.0
    f = O.ndft(x, C, 8)
    assert f[0, 0] == pytest.approx(cmath.exp(2j * math.pi * (1 * 0.1 - 4 * -0.2)))


def test_matern32_coeffs_equal_fourier_transform_3d():
    # Small ell: the kernel has decayed at the cell boundary ((1 + 17) e^-17
    # ~ 7e-7 at r = 1/2) and b_k approximates the continuous Fourier transform
    # of the remark in Sec. 4 (d = 3, nu = 3/2, l = sqrt(3) ell):
    #   kappa_hat(w) = 2^3 pi^{3/2} Gamma(3) 3^{3/2} / (Gamma(3/2) l^3)
    #                  * (3 / l^2 + 4 pi^2 |w|^2)^{-3}.
    N, ell = 64, 0.03
    l = math.sqrt(3.0) * ell
    b = O.fourier_coeffs("matern32", ell, N, 3)
    c = 2 ** 3 * math.pi ** 1.5 * math.gamma(3) * 3 ** 1.5 / (math.gamma(1.5) * l ** 3)
    for k in [(0, 0, 0), (1, 0, 0), (1, 2, 0), (3, 1, 2), (4, 4, 4)]:
        w2 = sum(t * t for t in k)
        want = c * (3.0 / l ** 2 + 4 * math.pi ** 2 * w2) ** -3
        got = b[tuple(t + N // 2 for t in k)].real
        assert got == pytest.approx(want, rel=2e-4), k
