"""Pins of the oracle's additive AFN preconditioner (Sec. 2.3): the FSAI
factor of the Schur complement against the textbook Cholesky inverse, the
exactness of the factorisation with a full pattern, the block identities of
M, the determinant and its derivative against dense linear algebra and
finite differences, the iteration saving of Sec. 5's first experiment, and
the pieces of the AFN-preconditioned likelihood estimate (dG and dM against
finite differences, the probe covariance, exactness with a full pattern,
agreement with a dense Hutchinson average over a full Krylov space)."""
import math

import numpy as np
import pytest

import oracle as O


def _problem(n=60, seed=70, ell=0.2, se=0.1):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-0.24, 0.24, size=(n, 4))
    W = [[0, 1], [2, 3]]
    th = dict(ell=ell, sigma_f=0.9, sigma_eps=se)
    L = O.additive_landmarks(X, W, 6)
    return X, W, th, L, rng


def _factors(X, W, th, L, fill, kind="gauss"):
    return O.afn_factors(X, W, kind, th["ell"], th["sigma_f"], th["sigma_eps"], L, fill)


def test_split_is_a_partition():
    L, F = O.afn_split(10, [7, 2, 2, 5])
    assert L == [2, 5, 7] and F == [0, 1, 3, 4, 6, 8, 9]


def test_pattern_holds_the_nearest_earlier_points():
    X, W, th, L, _ = _problem()
    fill = 7
    J = O.fsai_pattern(X, W, L, fill)
    _, F = O.afn_split(len(X), L)
    x = X[F]
    for t, Jt in enumerate(J):
        assert Jt[-1] == t and Jt == sorted(Jt) and len(set(Jt)) == len(Jt)
        assert len(Jt) == min(fill, t + 1)
        nb = Jt[:-1]
        if not nb:
            continue
        d = np.sum((x[:t] - x[t]) ** 2, axis=1)
        far = max(d[u] for u in nb)
        rest = [u for u in range(t) if u not in nb]
        # float64 distances; slack for the float32 decision
        assert all(d[u] >= far * (1 - 1e-5) for u in rest)


def test_fill_one_pattern_is_diagonal():
    X, W, th, L, _ = _problem()
    assert all(len(Jt) == 1 for Jt in O.fsai_pattern(X, W, L, 1))


def test_full_pattern_fsai_is_the_inverse_cholesky_factor():
    """With every earlier position in the pattern, the FSAI factor is the
    inverse of the lower Cholesky factor of S (textbook identity)."""
    X, W, th, L, _ = _problem(40)
    _, F, _, _, S, G, _ = _factors(X, W, th, L, fill=10 ** 6)
    np.testing.assert_allclose(G, np.linalg.inv(np.linalg.cholesky(S)), rtol=1e-8, atol=1e-10)


def test_full_pattern_preconditioner_is_the_matrix():
    X, W, th, L, _ = _problem(40)
    Lf, F, KLL, KFL, _, G, _ = _factors(X, W, th, L, fill=10 ** 6)
    M = O.afn_matrix(Lf, F, KLL, KFL, G)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    np.testing.assert_allclose(M, K, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("kind", ["gauss", "matern12"])
def test_fsai_defining_property_and_block_identities(kind):
    X, W, th, L, _ = _problem()
    Lf, F, KLL, KFL, S, G, J = _factors(X, W, th, L, fill=5, kind=kind)
    assert np.all(np.triu(G, 1) == 0)
    GS = G @ S
    for t, Jt in enumerate(J):
        assert abs(G[t] @ S @ G[t] - 1.0) < 1e-10
        for u in Jt[:-1]:
            assert abs(GS[t, u]) < 1e-10 * np.abs(GS[t]).max()
    M = O.afn_matrix(Lf, F, KLL, KFL, G)
    K = O.dense_matrix(X, W, kind, th["ell"], th["sigma_f"], th["sigma_eps"])
    # the landmark rows of M are those of K_hat; M is SPD
    np.testing.assert_allclose(M[Lf], K[Lf], rtol=1e-10, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > 0


def test_fill_one_keeps_the_diagonal():
    X, W, th, L, _ = _problem()
    Lf, F, KLL, KFL, S, G, _ = _factors(X, W, th, L, fill=1)
    np.testing.assert_allclose(np.diag(G), 1.0 / np.sqrt(np.diag(S)), rtol=1e-12)
    M = O.afn_matrix(Lf, F, KLL, KFL, G)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    np.testing.assert_allclose(np.diag(M), np.diag(K), rtol=1e-10)


def test_apply_inverse_and_logdet_match_dense():
    X, W, th, L, rng = _problem()
    Lf, F, KLL, KFL, _, G, _ = _factors(X, W, th, L, fill=5)
    M = O.afn_matrix(Lf, F, KLL, KFL, G)
    V = rng.standard_normal((len(X), 3))
    np.testing.assert_allclose(O.afn_apply_inverse(Lf, F, KLL, KFL, G, V),
                               np.linalg.solve(M, V), rtol=1e-8, atol=1e-9)
    _, ld = np.linalg.slogdet(M)
    assert abs(O.afn_logdet(KLL, G) - ld) < 1e-9 * abs(ld)


@pytest.mark.parametrize("which", ["ell", "sigma_f", "sigma_eps"])
def test_logdet_gradient_matches_finite_differences(which):
    X, W, th, L, _ = _problem(40)
    fill = 4

    def logdet(t):
        _, _, KLL, _, _, G, _ = _factors(X, W, t, L, fill)
        return O.afn_logdet(KLL, G)

    Lf, F, KLL, KFL, _, G, J = _factors(X, W, th, L, fill)
    g = O.afn_logdet_grad(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"],
                          Lf, F, KLL, KFL, G, J, which)
    h = 1e-5 * th[which]
    tp, tm = dict(th), dict(th)
    tp[which] += h
    tm[which] -= h
    fd = (logdet(tp) - logdet(tm)) / (2 * h)
    assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd)), (g, fd)


def test_afn_pcg_needs_fewer_iterations_than_cg():
    """Sec. 5 (first experiment, reduced): points uniform in a 6-D cube,
    sigma_f^2 = 1/P, sigma_eps^2 = 0.01, right-hand side uniform in
    [-0.5, 0.5], relative residual 1e-4. In the middle range of ell plain CG
    is slow and the AFN preconditioner cuts the iteration count."""
    rng = np.random.default_rng(5)
    n = 400
    X = rng.uniform(-0.24, 0.24, size=(n, 6))
    W = [[0, 1, 2], [3, 4, 5]]
    sf, se, ell = math.sqrt(0.5), 0.1, 0.15
    K = O.dense_matrix(X, W, "matern12", ell, sf, se)
    b = rng.uniform(-0.5, 0.5, size=(n, 1))
    L = O.additive_landmarks(X, W, 60)
    Lf, F, KLL, KFL, _, G, _ = O.afn_factors(X, W, "matern12", ell, sf, se, L, 20)
    _, it_cg, _, _, _ = O.cg(lambda P: K @ P, b, rtol=1e-4, maxit=400)
    xs, it_p, rel = O.pcg(lambda P: K @ P,
                          lambda P: O.afn_apply_inverse(Lf, F, KLL, KFL, G, P), b,
                          rtol=1e-4, maxit=400)
    assert rel[0] <= 1e-4
    assert np.linalg.norm(K @ xs - b) <= 1.01e-4 * np.linalg.norm(b)
    assert it_p[0] < 0.5 * it_cg[0], (it_p, it_cg)


def _fd(f, th, which, h_rel=1e-5):
    h = h_rel * th[which]
    tp, tm = dict(th), dict(th)
    tp[which] += h
    tm[which] -= h
    return (f(tp) - f(tm)) / (2 * h)


@pytest.mark.parametrize("which", ["ell", "sigma_f", "sigma_eps"])
def test_dG_and_dM_match_finite_differences(which):
    X, W, th, L, _ = _problem(36)
    fill = 5
    Lf, F, KLL, KFL, S, G, J = _factors(X, W, th, L, fill)
    args = (X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"], Lf, F, KLL, KFL, S, G, J,
            which)
    dG = O.afn_dG(*args)
    fdG = _fd(lambda t: _factors(X, W, t, L, fill)[5], th, which)
    np.testing.assert_allclose(dG, fdG, rtol=1e-5, atol=1e-6 * np.abs(fdG).max())

    def M_of(t):
        a = _factors(X, W, t, L, fill)
        return O.afn_matrix(a[0], a[1], a[2], a[3], a[5])

    dM = O.afn_dM(*args)
    fdM = _fd(M_of, th, which)
    np.testing.assert_allclose(dM, fdM, rtol=1e-5, atol=1e-6 * np.abs(fdM).max())
    # and its trace against the log-determinant derivative
    M = M_of(th)
    tr = float(np.trace(np.linalg.solve(M, dM)))
    g = O.afn_logdet_grad(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"], Lf, F, KLL, KFL,
                          G, J, which)
    assert abs(tr - g) <= 1e-8 * max(1.0, abs(g))


def test_probes_have_covariance_M():
    X, W, th, L, _ = _problem(30)
    Lf, F, KLL, KFL, _, G, _ = _factors(X, W, th, L, fill=4)
    Z = O.afn_probes(Lf, F, KLL, KFL, G, np.eye(30))
    np.testing.assert_allclose(Z @ Z.T, O.afn_matrix(Lf, F, KLL, KFL, G), rtol=1e-10, atol=1e-12)


def test_afn_estimate_with_full_pattern_is_exact():
    """fill >= n - k: M = K_hat, so M^{-1} K_hat = I, every SLQ term vanishes,
    p_i = u_i and dM = dK_hat: the estimate is the exact NLML and gradient
    whatever the probes."""
    X, W, th, L, rng = _problem(40)
    n = len(X)
    y = rng.standard_normal(n)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    dK = {w: O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"], which=w)
          for w in ("ell", "sigma_f", "sigma_eps")}
    nl, g = O.nlml_estimate_afn(lambda P: K @ P, {w: (lambda P, A=A: A @ P) for w, A in dK.items()},
                                y, rng.standard_normal((n, 5)), 6, X, W, "gauss", th["ell"],
                                th["sigma_f"], th["sigma_eps"], L, 10 ** 6)
    assert abs(nl - O.nlml_exact(K, y)) <= 1e-9 * abs(nl)
    a = np.linalg.solve(K, y)
    for w, A in dK.items():
        exact = 0.5 * (-(a @ A @ a) + np.trace(np.linalg.solve(K, A)))
        assert abs(g[w] - exact) <= 1e-8 * max(1.0, abs(exact)), (w, g[w], exact)


def test_afn_estimate_with_full_krylov_space_is_hutchinson():
    """With as many PCG steps as points each SLQ term is exact, so the
    estimate equals log det M + the Hutchinson average of z~^T log(M^{-1/2}
    K_hat M^{-1/2}) z~ (z~ = M^{-1/2} z), from a dense eigendecomposition."""
    X, W, th, L, rng = _problem(24)
    n = len(X)
    fill = 3
    y = rng.standard_normal(n)
    Wn = rng.standard_normal((n, 4))
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    nl, _ = O.nlml_estimate_afn(lambda P: K @ P, {}, y, Wn, n, X, W, "gauss", th["ell"],
                                th["sigma_f"], th["sigma_eps"], L, fill)
    Lf, F, KLL, KFL, _, G, _ = _factors(X, W, th, L, fill)
    M = O.afn_matrix(Lf, F, KLL, KFL, G)
    ew, V = np.linalg.eigh(M)
    Mh = V @ np.diag(ew ** -0.5) @ V.T
    ew2, V2 = np.linalg.eigh(Mh @ K @ Mh)
    logm = V2 @ np.diag(np.log(ew2)) @ V2.T
    Zt = Mh @ O.afn_probes(Lf, F, KLL, KFL, G, Wn)
    quad = np.mean(np.sum(Zt * (logm @ Zt), axis=0))
    want = 0.5 * (y @ np.linalg.solve(K, y) + O.afn_logdet(KLL, G) + quad + n * math.log(2 * math.pi))
    assert abs(nl - want) <= 1e-7 * abs(want)
