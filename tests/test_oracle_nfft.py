"""Pins of the oracle's NFFT (Appendix A): the Kaiser-Bessel window and its
Fourier transform against quadrature, and the NFFT and its adjoint against the
exact NDFT within the window error bound printed in Appendix A."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import oracle as O


def test_kb_window_closed_values():
    s, n_os = 4, 64
    b = 1.5 * math.pi
    assert O.kb_window(0.0, n_os, s) == pytest.approx(math.sinh(b * s) / (math.pi * s), rel=1e-14)
    assert O.kb_window(s / n_os, n_os, s) == pytest.approx(b / math.pi, rel=1e-12)
    assert O.kb_window(s / n_os * 1.001, n_os, s) == 0.0


@pytest.mark.parametrize("n_os,s", [(64, 4), (64, 5), (128, 5), (32, 3)])
def test_kb_window_hat_matches_quadrature(n_os, s):
    # phi_hat(k) = int phi(x) e^{-2 pi i k x} dx over the truncated support.
    # The closed form is the transform of the untruncated window, whose tail
    # beyond the support is bounded by b/pi, so the two differ relatively by
    # O(1 / I0(b s)).
    rel = max(1e-10, 20.0 / scipy.special.i0(1.5 * math.pi * s))
    for k in [0, 1, 5, n_os // 4]:
        f = lambda x: O.kb_window(x, n_os, s) * math.cos(2 * math.pi * k * x)
        q, _ = scipy.integrate.quad(f, -s / n_os, s / n_os, epsabs=0, epsrel=1e-13, limit=200)
        assert O.kb_window_hat(k, n_os, s) == pytest.approx(q, rel=rel)


def test_bins_floor():
    x = np.array([-0.25, -0.2500001, 0.0, -1e-9, 0.2499999, 1 / 64])
    np.testing.assert_array_equal(O.bins(x, 64), [-16, -17, 0, -1, 15, 1])


def _bound(s, sigma, d):
    # Appendix A eq. (A.2) (per unit l1 norm), with the d-dimensional
    # constant growing like d 2^{d-1}.
    one = 4 * math.pi * (s + math.sqrt(s)) * (1 - 1 / sigma) ** 0.25 \
        * math.exp(-2 * math.pi * s * math.sqrt(1 - 1 / sigma))
    return one * d * 2 ** (d - 1)


@pytest.mark.parametrize("d,N,s", [(1, 32, 4), (2, 16, 4), (3, 8, 3), (2, 16, 2)])
def test_nfft_within_window_error_bound(d, N, s):
    rng = np.random.default_rng(20 + d)
    x = rng.uniform(-0.25, 0.25, size=(60, d))
    C = rng.standard_normal((N,) * d + (1,)) + 1j * rng.standard_normal((N,) * d + (1,))
    C /= np.sum(np.abs(C))
    err = np.max(np.abs(O.nfft(x, C, N, s) - O.ndft(x, C, N)))
    assert err <= _bound(s, 2.0, d)
    assert err > 0          # the NFFT is an approximation, not the NDFT itself


@pytest.mark.parametrize("d,N,s", [(1, 32, 4), (2, 16, 4), (3, 8, 3)])
def test_nfft_adjoint_within_window_error_bound(d, N, s):
    rng = np.random.default_rng(30 + d)
    x = rng.uniform(-0.25, 0.25, size=(50, d))
    v = rng.standard_normal((50, 2))
    err = np.max(np.abs(O.nfft_adjoint(x, v, N, s) - O.ndft_adjoint(x, v, N)))
    assert err <= _bound(s, 2.0, d) * np.max(np.sum(np.abs(v), axis=0))


@pytest.mark.parametrize("kind", ["gauss", "matern12"])
def test_nfft_fastsum_matches_truncated_sum(kind):
    rng = np.random.default_rng(40)
    X = rng.uniform(-0.24, 0.24, size=(150, 5))
    v = rng.standard_normal((150, 2))
    W = [[0, 1, 2], [3, 4]]
    a = O.nfft_fastsum_matvec(X, W, kind, 0.3, 1.0, 0.1, v, 16, 5)
    b = O.truncated_matvec(X, W, kind, 0.3, 1.0, 0.1, v, 16)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8
