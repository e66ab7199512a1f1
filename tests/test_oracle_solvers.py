"""Pins of the oracle's CG, SLQ and likelihood (Sec. 1) to dense linear algebra
and to scipy's multivariate normal density."""
import math

import numpy as np
import pytest
import scipy.stats

import oracle as O


def _problem(n=12, seed=50):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-0.24, 0.24, size=(n, 4))
    W = [[0, 1], [2, 3]]
    th = dict(ell=0.2, sigma_f=0.9, sigma_eps=0.6)
    return X, W, th, rng


def test_cg_matches_cholesky_solve():
    X, W, th, rng = _problem(40)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    B = rng.standard_normal((40, 3))
    Xs, it, rel, _, _ = O.cg(lambda P: K @ P, B, rtol=1e-12, maxit=400)
    np.testing.assert_allclose(Xs, np.linalg.solve(K, B), rtol=1e-8, atol=1e-9)
    assert np.all(rel <= 1e-12) and np.all(it > 0)


def test_cg_zero_rhs_and_iteration_cap():
    X, W, th, rng = _problem(30)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], 0.01)
    B = np.zeros((30, 2))
    B[:, 1] = rng.standard_normal(30)
    Xs, it, rel, _, _ = O.cg(lambda P: K @ P, B, rtol=1e-14, maxit=3)
    assert it[0] == 0 and rel[0] == 0 and np.all(Xs[:, 0] == 0)
    assert it[1] == 3 and rel[1] > 1e-14


def test_pcg_with_identity_is_cg_and_matches_solve():
    X, W, th, rng = _problem(40)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    B = rng.standard_normal((40, 2))
    Xp, itp, _ = O.pcg(lambda P: K @ P, lambda P: P, B, rtol=1e-12, maxit=400)
    Xc, itc, _, _, _ = O.cg(lambda P: K @ P, B, rtol=1e-12, maxit=400)
    np.testing.assert_array_equal(itp, itc)
    np.testing.assert_allclose(Xp, Xc, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Xp, np.linalg.solve(K, B), rtol=1e-8, atol=1e-9)


def test_farthest_point_sampling_brute_force():
    # each chosen point has the largest distance to the points chosen before
    # it (checked by enumeration), the first is index 0, and a duplicate of an
    # earlier point is never chosen while a farther point exists
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.24, 0.24, size=(60, 2))
    x[17] = x[0]
    ch = O.farthest_point_sampling(x, 12)
    assert ch[0] == 0 and len(set(ch)) == 12 and 17 not in ch
    for t in range(1, 12):
        prev = x[ch[:t]]
        md = [min(np.sum((x[i] - p) ** 2) for p in prev) for i in range(60)]
        assert md[ch[t]] == pytest.approx(max(md), rel=1e-6)
    # three points on a line: 0, then the far end, then the middle
    line = np.array([[0.0], [0.1], [0.2]])
    assert O.farthest_point_sampling(line, 3) == [0, 2, 1]


def test_nystrom_with_all_points_is_exact():
    # L = every point: K_{:,L} K_LL^{-1} K_{L,:} = K, so M = K_hat and one PCG
    # step solves the system
    X, W, th, rng = _problem(30)
    K = O.dense_matrix(X, W, "matern12", th["ell"], th["sigma_f"], th["sigma_eps"])
    Minv = O.nystrom_preconditioner(X, W, "matern12", th["ell"], th["sigma_f"], th["sigma_eps"],
                                    range(30), jitter=0.0)
    B = rng.standard_normal((30, 2))
    np.testing.assert_allclose(Minv(B), np.linalg.solve(K, B), rtol=1e-6, atol=1e-8)
    Xs, it, _ = O.pcg(lambda P: K @ P, Minv, B, rtol=1e-8, maxit=5)
    assert np.all(it == 1)


def test_additive_landmarks_union_per_window():
    rng = np.random.default_rng(4)
    X = rng.uniform(-0.24, 0.24, size=(80, 5))
    W = [[0, 1, 2], [3, 4]]
    L = O.additive_landmarks(X, W, 7)
    want = sorted(set(O.farthest_point_sampling(X[:, [0, 1, 2]], 4)) |
                  set(O.farthest_point_sampling(X[:, [3, 4]], 4)))
    assert L == want and L[0] == 0


def test_slq_exact_with_full_krylov_space():
    # With as many Lanczos steps as the dimension, Gauss quadrature is exact:
    # z^T logm(A) z = |z|^2 sum tau^2 log theta.
    X, W, th, rng = _problem(12)
    K = O.dense_matrix(X, W, "gauss", th["ell"], th["sigma_f"], th["sigma_eps"])
    lam, Q = np.linalg.eigh(K)
    logK = (Q * np.log(lam)) @ Q.T
    z = rng.choice([-1.0, 1.0], size=12)
    _, _, _, al, be = O.cg(lambda P: K @ P, z[:, None], fixed_iters=12)
    T = O.lanczos_tridiag_from_cg(al[0], be[0])
    assert O.slq_quadratic(T, z @ z) == pytest.approx(z @ logK @ z, rel=1e-9)


def test_slq_breakdown_ends_the_lanczos_matrix_at_an_invariant_subspace():
    # A well-conditioned matrix whose CG residual reaches 1e-12 in far fewer
    # steps than its dimension: with the breakdown floor the recursion stops
    # there and the quadrature equals z^T logm(A) z (eigendecomposition) to
    # rounding level, however many steps are asked for; the steps it would
    # take past that point only divide rounding-level residual norms.
    rng = np.random.default_rng(5)
    n = 200
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 1.5, n)
    A = (Q * lam) @ Q.T
    z = rng.choice([-1.0, 1.0], size=n)
    want = z @ ((Q * np.log(lam)) @ Q.T) @ z
    for steps in (40, 120):
        _, it, rel, al, be = O.cg(lambda P: A @ P, z[:, None], fixed_iters=steps,
                                  breakdown=O.LANCZOS_BREAKDOWN)
        assert it[0] < 40 and rel[0] <= O.LANCZOS_BREAKDOWN
        T = O.lanczos_tridiag_from_cg(al[0], be[0])
        assert O.slq_quadratic(T, z @ z) == pytest.approx(want, rel=1e-10)


def test_nlml_exact_matches_scipy_logpdf():
    X, W, th, rng = _problem(25)
    K = O.dense_matrix(X, W, "matern12", th["ell"], th["sigma_f"], th["sigma_eps"])
    y = rng.standard_normal(25)
    want = -scipy.stats.multivariate_normal(mean=np.zeros(25), cov=K).logpdf(y)
    assert O.nlml_exact(K, y) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("kind", ["gauss", "matern12"])
def test_nlml_estimate_exact_with_orthogonal_probes(kind):
    # Probes sqrt(n) q_i from an orthogonal basis make Hutchinson exact, and n
    # Lanczos steps make each quadrature exact, so the estimator must return
    # the exact NLML and the exact gradient (finite differences of scipy's
    # log density).
    n = 12
    X, W, th, rng = _problem(n)
    y = rng.standard_normal(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Z = math.sqrt(n) * Q

    def Kmat(**kw):
        t = dict(th, **kw)
        return O.dense_matrix(X, W, kind, t["ell"], t["sigma_f"], t["sigma_eps"])

    K = Kmat()
    dK = {w: O.dense_matrix(X, W, kind, th["ell"], th["sigma_f"], th["sigma_eps"], which=w)
          for w in ["ell", "sigma_f", "sigma_eps"]}
    nl, g = O.nlml_estimate(lambda P: K @ P, {w: (lambda P, M=M: M @ P) for w, M in dK.items()},
                            y, Z, lanczos_steps=n)

    def Zexact(**kw):
        return -scipy.stats.multivariate_normal(mean=np.zeros(n), cov=Kmat(**kw)).logpdf(y)

    assert nl == pytest.approx(Zexact(), rel=1e-8)
    h = 1e-6
    for w in ["ell", "sigma_f", "sigma_eps"]:
        fd = (Zexact(**{w: th[w] + h}) - Zexact(**{w: th[w] - h})) / (2 * h)
        assert g[w] == pytest.approx(fd, rel=1e-5, abs=1e-7)


# ---------------------------------------------------------------------------
# preconditioned estimator (Sec. 1 eqs. (1.3)-(1.5) with the landmark M)
# ---------------------------------------------------------------------------
def _nystrom_problem(n=12, k_total=4, kind="matern12", seed=60):
    X, W, th, rng = _problem(n, seed)
    L = O.additive_landmarks(X, W, k_total)
    return X, W, th, rng, L


@pytest.mark.parametrize("kind", ["gauss", "matern12"])
def test_nystrom_logdet_matches_dense(kind):
    X, W, th, _, L = _nystrom_problem(kind=kind)
    B, KLL = O.nystrom_blocks(X, W, kind, th["ell"], th["sigma_f"], L, sigma_eps=th["sigma_eps"])
    s2 = th["sigma_eps"] ** 2
    _, want = np.linalg.slogdet(O.nystrom_matrix(B, KLL, s2))
    assert O.nystrom_logdet(B, KLL, s2) == pytest.approx(want, rel=1e-11)


def test_nystrom_probes_have_covariance_M():
    # with w_i = sqrt(n+k) q_i over an orthogonal basis of R^{n+k}, the mean
    # of z_i z_i^T is F F^T = M exactly
    X, W, th, rng, L = _nystrom_problem()
    B, KLL = O.nystrom_blocks(X, W, "matern12", th["ell"], th["sigma_f"], L,
                              sigma_eps=th["sigma_eps"])
    n, k = B.shape
    Q, _ = np.linalg.qr(rng.standard_normal((n + k, n + k)))
    Wf = math.sqrt(n + k) * Q
    Z = O.nystrom_probes(B, KLL, th["sigma_eps"], Wf[:n], Wf[n:])
    M = O.nystrom_matrix(B, KLL, th["sigma_eps"] ** 2)
    np.testing.assert_allclose(Z @ Z.T / (n + k), M, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("which", ["ell", "sigma_f"])
def test_nystrom_dM_terms_match_finite_differences(which):
    # tr(M^{-1} dM) = d/dtheta log det M and p^T dM p = d/dtheta p^T M p,
    # each against central differences of M(theta) built from scratch
    X, W, th, rng, L = _nystrom_problem(kind="gauss")
    s2 = th["sigma_eps"] ** 2
    B, KLL = O.nystrom_blocks(X, W, "gauss", th["ell"], th["sigma_f"], L, sigma_eps=th["sigma_eps"])
    dB, _ = O.nystrom_blocks(X, W, "gauss", th["ell"], th["sigma_f"], L, which=which)
    dKLL = dB[L]
    h = 1e-5

    jit = O.landmark_jitter(B, B[L], th["sigma_f"], len(W), th["sigma_eps"])   # fixed, as in dM

    def at(delta):
        t = dict(th)
        t[which] += delta
        Bh, Kh = O.nystrom_blocks(X, W, "gauss", t["ell"], t["sigma_f"], L, jitter=jit)
        return O.nystrom_matrix(Bh, Kh, s2), O.nystrom_logdet(Bh, Kh, s2)

    (Mp, lp), (Mm, lm) = at(h), at(-h)
    assert O.nystrom_trace_Minv_dM(B, KLL, dB, dKLL, s2) == pytest.approx((lp - lm) / (2 * h),
                                                                           rel=1e-6)
    P = rng.standard_normal((X.shape[0], 3))
    fd = np.sum(P * ((Mp - Mm) / (2 * h) @ P), axis=0)
    np.testing.assert_allclose(O.nystrom_dM_quadratic(B, KLL, dB, dKLL, P), fd, rtol=1e-6)


@pytest.mark.parametrize("kind", ["gauss", "matern12"])
def test_nlml_preconditioned_exact_with_orthogonal_probes(kind):
    # probes over a scaled orthogonal basis of R^{n+k} (so mean z z^T = M) and
    # n-k+1 PCG steps (M^{-1} K_hat has eigenvalue 1 with multiplicity >= k,
    # hence at most n-k+1 distinct eigenvalues) make the estimator exact: it
    # must return scipy's NLML and its finite-difference gradient
    n = 12
    X, W, th, rng, L = _nystrom_problem(n, 4, kind)
    k = len(L)
    y = rng.standard_normal(n)
    B, KLL = O.nystrom_blocks(X, W, kind, th["ell"], th["sigma_f"], L, sigma_eps=th["sigma_eps"])
    dB = {w: O.nystrom_blocks(X, W, kind, th["ell"], th["sigma_f"], L, which=w)[0]
          for w in ["ell", "sigma_f"]}
    Q, _ = np.linalg.qr(rng.standard_normal((n + k, n + k)))
    Wf = math.sqrt(n + k) * Q

    def Kmat(**kw):
        t = dict(th, **kw)
        return O.dense_matrix(X, W, kind, t["ell"], t["sigma_f"], t["sigma_eps"])

    K = Kmat()
    dK = {w: O.dense_matrix(X, W, kind, th["ell"], th["sigma_f"], th["sigma_eps"], which=w)
          for w in ["ell", "sigma_f", "sigma_eps"]}
    nl, g = O.nlml_estimate_preconditioned(
        lambda P: K @ P, {w: (lambda P, M=M: M @ P) for w, M in dK.items()}, y, Wf[:n], Wf[n:],
        n - k + 1, B, KLL, dB, L, th["sigma_eps"])

    def Zexact(**kw):
        return -scipy.stats.multivariate_normal(mean=np.zeros(n), cov=Kmat(**kw)).logpdf(y)

    assert nl == pytest.approx(Zexact(), rel=1e-8)
    h = 1e-6
    for w in ["ell", "sigma_f", "sigma_eps"]:
        fd = (Zexact(**{w: th[w] + h}) - Zexact(**{w: th[w] - h})) / (2 * h)
        assert g[w] == pytest.approx(fd, rel=1e-5, abs=1e-7), w


def test_splitmix64_published_vectors():
    # the first outputs of SplitMix64 from state 0, as printed by the
    # generator's reference implementation (Steele, Lea and Flood, OOPSLA
    # 2014; the splitmix64.c of Vigna's xorshift/xoroshiro distribution)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in O.splitmix64(0, 4)] == want
    # counter-based: output i of seed s is output i + 1 of seed s - g
    g = 0x9E3779B97F4A7C15
    a = O.splitmix64(12345, 10)
    b = O.splitmix64((12345 - g) % (1 << 64), 11)
    assert [int(v) for v in a] == [int(v) for v in b[1:]]


def test_rademacher_probes_signs_and_balance():
    Z = O.rademacher_probes(20000, 7, 99)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 0.02
    # entry (i, c) is output i R + c: the top bit decides the sign
    z = O.splitmix64(99, 20000 * 7)
    assert Z[3, 5] == (1.0 if int(z[3 * 7 + 5]) >> 63 == 0 else -1.0)
