"""GPU parity of the additive AFN preconditioner (Sec. 2.3): landmarks and the
FSAI pattern index for index, M^{-1} and log det M against the oracle's dense
construction (both FP64 from the same coordinates), the block identities at
a size the oracle cannot factorise densely, and PCG with it."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_00480_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]
DEV = "cuda:0"


@pytest.fixture(scope="module")
def agp():
    from paper_2504_00480_gb300 import agp as A
    from paper_2504_00480_gb300 import build
    build.build()
    A.load_library()
    return A


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def points(n, p, seed, dtype):
    rng = np.random.default_rng(seed)
    X = inputs.minmax_scale(rng.uniform(-1.0, 1.0, size=(n, p)))
    if n > 60:
        X[50] = X[40]            # an exact duplicate: a zero distance
    return inputs.to_precision(X, dtype).astype(np.float64), rng


def compare_pattern(J, want, rows, rel_bound=1e-12):
    """Rows of the device pattern against the oracle's (J_t, gap_t): equal,
    with -1 after the row's entries, except rows whose deciding gap is a
    near-tie (positive, below rel_bound x the distance scale), which are
    skipped and counted. Returns the number of skipped rows."""
    skipped = 0
    for t, (Jt, gap) in zip(rows, want):
        if 0.0 < gap <= rel_bound:
            skipped += 1
            continue
        row = J[t]
        assert list(row[:len(Jt)]) == Jt and np.all(row[len(Jt):] == -1), t
    return skipped


def make(agp, X, W, dtype, kind, th, N=32, s=5):
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    return agp.Plan(torch.tensor(X, dtype=tdt, device=DEV), W, N, s, kind, *th)


CASES = [(np.float64, "gauss", (0.15, 0.9, 0.1)), (np.float32, "matern12", (0.2, 1.0, 0.1)),
         (np.float64, "matern32", (0.1, 0.8, 0.2))]


@pytest.mark.parametrize("dtype,kind,th", CASES)
@pytest.mark.parametrize("fill", [1, 7, 40])
def test_pattern_inverse_and_logdet_match_oracle(agp, dtype, kind, th, fill):
    X, rng = points(700, 5, 11, dtype)
    W = [[0, 1, 2], [3, 4]]
    plan = make(agp, X, W, dtype, kind, th)
    afn = plan.afn(24, fill)
    lm, J = afn.pattern()
    want_lm = O.additive_landmarks(X, W, 24)
    np.testing.assert_array_equal(lm, want_lm)
    want = O.fsai_pattern_gaps(X, W, want_lm, fill)
    want_J = [Jt for Jt, _ in want]
    skipped = compare_pattern(J, want, range(len(want)))
    assert skipped <= len(want) // 100, skipped
    L, F, KLL, KFL, _, G, _ = O.afn_factors(X, W, kind, *th, want_lm, fill)
    V = rng.standard_normal((len(X), 6))
    got = afn.apply(torch.tensor(V, device=DEV)).cpu().numpy()
    want = O.afn_apply_inverse(L, F, KLL, KFL, G, V)
    assert rel(got, want) <= 1e-9
    k, nnz, logdet = afn.info()
    assert k == len(L) and nnz == sum(len(Jt) for Jt in want_J)
    assert abs(logdet - O.afn_logdet(KLL, G)) <= 1e-10 * abs(logdet) + 1e-9


def test_full_pattern_gives_the_exact_inverse(agp):
    """With fill above the number of non-landmark points every row of G holds
    all earlier positions, G is the inverse Cholesky factor of S and M = K_hat."""
    X, rng = points(100, 4, 12, np.float64)
    W = [[0, 1], [2, 3]]
    th = (0.2, 1.0, 0.1)
    plan = make(agp, X, W, np.float64, "gauss", th)
    afn = plan.afn(8, 128)
    V = rng.standard_normal((100, 2))
    got = afn.apply(torch.tensor(V, device=DEV)).cpu().numpy()
    K = O.dense_matrix(X, W, "gauss", *th)
    assert rel(got, np.linalg.solve(K, V)) <= 1e-9
    assert abs(afn.info()[2] - np.linalg.slogdet(K)[1]) <= 1e-9 * abs(np.linalg.slogdet(K)[1])


def test_all_points_are_landmarks(agp):
    """n <= landmarks per window: the Schur complement is empty and M = K_hat."""
    X, rng = points(8, 4, 13, np.float64)
    W = [[0, 1], [2, 3]]
    th = (0.3, 1.0, 0.2)
    plan = make(agp, X, W, np.float64, "gauss", th, N=16, s=4)
    afn = plan.afn(16, 4)
    k, nnz, logdet = afn.info()
    assert k == 8 and nnz == 0
    K = O.dense_matrix(X, W, "gauss", *th)
    V = rng.standard_normal((8, 3))
    got = afn.apply(torch.tensor(V, device=DEV)).cpu().numpy()
    assert rel(got, np.linalg.solve(K, V)) <= 1e-10
    assert abs(logdet - np.linalg.slogdet(K)[1]) <= 1e-10 * abs(logdet)


def test_large_fp32_block_identity_and_sampled_pattern(agp):
    """n = 60,000 (FP32 plan, 3 windows): sampled pattern rows against the
    oracle, and the landmark rows of M equal those of K_hat, so for y = M^{-1} v
    the landmark rows of K_hat y must reproduce v (checked with the oracle's
    exact dense rows)."""
    n = 60_000
    X, rng = points(n, 8, 14, np.float32)
    W = [[0, 1, 2], [3, 4, 5], [6, 7]]
    th = (0.1, 0.7, 0.1)
    plan = make(agp, X, W, np.float32, "gauss", th)
    afn = plan.afn(30, 50)
    lm, J = afn.pattern()
    np.testing.assert_array_equal(lm, O.additive_landmarks(X, W, 30))
    sample = [0, 1, 2, 49, 50, 51, 1234, 30_000, n - len(lm) - 1]
    want = O.fsai_pattern_gaps(X, W, lm, 50, rows=sample)
    assert compare_pattern(J, want, sample) == 0
    V = rng.standard_normal((n, 4))
    Y = afn.apply(torch.tensor(V, device=DEV)).cpu().numpy()
    KY = O.dense_matvec(X, W, "gauss", *th, Y, rows=lm)
    assert rel(KY, V[lm]) <= 1e-9


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pcg_with_afn_follows_oracle_and_beats_cg(agp, dtype):
    """Sec. 5's first experiment, reduced: points uniform in a 6-D cube,
    sigma_f^2 = 1/P, sigma_eps^2 = 0.01, right-hand side uniform in
    [-0.5, 0.5], relative residual 1e-4; Matern(1/2) in the middle range of ell."""
    n = 1500
    rng = np.random.default_rng(21)
    X = inputs.to_precision(rng.uniform(-0.24, 0.24, size=(n, 6)), dtype).astype(np.float64)
    W = [[0, 1, 2], [3, 4, 5]]
    th = (0.15, math.sqrt(0.5), 0.1)
    plan = make(agp, X, W, dtype, "matern12", th)
    b = rng.uniform(-0.5, 0.5, size=(n, 1))
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    B = torch.tensor(b, dtype=tdt, device=DEV)
    afn = plan.afn(100, 30)
    x_p, it_p, rel_p = afn.solve(B, rtol=1e-4, maxit=400)
    _, it_c, _ = plan.solve(B, rtol=1e-4, maxit=400)
    assert rel_p[0] <= 1e-4 and it_p[0] < 0.6 * it_c[0], (it_p, it_c)
    # the oracle's PCG on the Fourier-truncated operator with the oracle's M
    lm = O.additive_landmarks(X, W, 100)
    L, F, KLL, KFL, _, G, _ = O.afn_factors(X, W, "matern12", *th, lm, 30)

    def A(P):
        return O.truncated_matvec(X, W, "matern12", *th, P, 32)

    _, it_o, _ = O.pcg(A, lambda P: O.afn_apply_inverse(L, F, KLL, KFL, G, P), b,
                       rtol=1e-4, maxit=400)
    assert abs(int(it_p[0]) - int(it_o[0])) <= max(2, 0.15 * it_o[0]), (it_p, it_o)
    r = b - A(x_p.double().cpu().numpy())
    assert np.linalg.norm(r) <= 2e-4 * np.linalg.norm(b)


def test_rejects_bad_arguments_and_stale_hyperparameters(agp):
    X, _ = points(200, 4, 15, np.float64)
    W = [[0, 1], [2, 3]]
    plan = make(agp, X, W, np.float64, "gauss", (0.2, 1.0, 0.1))
    for k, fill in ((0, 5), (481, 5), (10, 0), (10, 129)):
        with pytest.raises(agp.AgpError):
            plan.afn(k, fill)
    afn = plan.afn(10, 5)
    plan.set_hyper(0.25, 1.0, 0.1)
    B = torch.ones((200, 1), dtype=torch.float64, device=DEV)
    with pytest.raises(agp.AgpError):
        afn.solve(B)
    noiseless = make(agp, X, W, np.float64, "gauss", (0.2, 1.0, 0.0))
    with pytest.raises(agp.AgpError):
        noiseless.afn(10, 5)


def _o2_dense(X, W, kind, ell, sf, se, N, which=None):
    """The Fourier-truncated operator (or a derivative) as a dense matrix."""
    n = X.shape[0]
    M = np.zeros((n, n))
    for a in range(0, n, 250):
        E = np.zeros((n, min(250, n - a)))
        E[np.arange(a, a + E.shape[1]), np.arange(E.shape[1])] = 1.0
        if which is None:
            M[:, a:a + E.shape[1]] = O.truncated_matvec(X, W, kind, ell, sf, se, E, N)
        else:
            M[:, a:a + E.shape[1]] = O.truncated_deriv_matvec(X, W, kind, ell, sf, se, E, N, which)
    return 0.5 * (M + M.T)


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-7), (np.float32, 2e-3)])
def test_nlml_afn_matches_oracle_estimator(agp, dtype, tol):
    """Same landmarks, pattern, probe vectors and step count: the GPU
    estimator against the oracle's (Fourier-truncated operator, exact-kernel
    AFN preconditioner, probes z = Phi [C w_L; G^{-1} w_F])."""
    n = 1000
    rng = np.random.default_rng(9)
    X = inputs.to_precision(inputs.minmax_scale(rng.standard_normal((n, 4))), dtype).astype(np.float64)
    W = [[0, 1], [2, 3]]
    th = ("gauss", 0.08, 1.0, 0.3)
    K = _o2_dense(X, W, *th, 32)
    dK = {w: _o2_dense(X, W, *th, 32, w) for w in ["ell", "sigma_f", "sigma_eps"]}
    plan = make(agp, X, W, dtype, th[0], th[1:])
    L = O.additive_landmarks(X, W, 40)
    nz, steps, fill = 6, 10, 10
    y = rng.standard_normal(n)
    Wn = inputs.to_precision(rng.standard_normal((n, nz)), dtype).astype(np.float64)
    nl_o, g_o = O.nlml_estimate_afn(lambda P: K @ P, {w: (lambda P, A=A: A @ P) for w, A in dK.items()},
                                    y, Wn, steps, X, W, *th, L, fill, rtol=0, maxit=steps)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    afn = plan.afn(40, fill)
    nl, g = afn.nlml_grad(torch.tensor(y, dtype=tdt, device=DEV),
                          torch.tensor(Wn, dtype=tdt, device=DEV), lanczos_steps=steps)
    assert nl == pytest.approx(nl_o, rel=tol)
    for w in g:
        assert g[w] == pytest.approx(g_o[w], rel=10 * tol, abs=10 * tol * abs(nl_o) / n), w


def test_nlml_afn_cuts_the_estimator_variance(agp):
    """Sec. 5 (second experiment, reduced): over several probe sets the
    AFN-preconditioned estimates of the NLML and of dZ/dell scatter far less
    than the unpreconditioned ones and centre on the exact values (dense
    Cholesky of the truncated operator)."""
    n = 800
    rng = np.random.default_rng(23)
    X = rng.uniform(-0.24, 0.24, size=(n, 6))
    W = [[0, 1, 2], [3, 4, 5]]
    th = ("matern12", 0.2, math.sqrt(0.5), 0.1)
    K = _o2_dense(X, W, *th, 32)
    dKl = _o2_dense(X, W, *th, 32, "ell")
    y = rng.standard_normal(n)
    exact = O.nlml_exact(K, y)
    a = np.linalg.solve(K, y)
    exact_dl = 0.5 * (-(a @ dKl @ a) + np.trace(np.linalg.solve(K, dKl)))
    plan = make(agp, X, W, np.float64, th[0], th[1:])
    afn = plan.afn(100, 30)
    yt = torch.tensor(y, device=DEV)
    pc, pl = [], []
    for s in range(6):
        r = np.random.default_rng(1000 + s)
        Wn = torch.tensor(r.standard_normal((n, 5)), device=DEV)
        nl, g = afn.nlml_grad(yt, Wn, lanczos_steps=10, rtol=1e-10, maxit=2000)
        pc.append((nl, g["ell"]))
        Z = torch.tensor(inputs.rademacher(n, 5, 2000 + s), device=DEV)
        nl, g = plan.nlml_grad(yt, Z, lanczos_steps=10, rtol=1e-10, maxit=2000)
        pl.append((nl, g["ell"]))
    pc, pl = np.array(pc), np.array(pl)
    # the oracle on the same probes: std 3.4 vs 8.8 (NLML), 2.8 vs 16 (dZ/dell)
    assert pc[:, 0].std() < 0.6 * pl[:, 0].std() and pc[:, 1].std() < 0.3 * pl[:, 1].std()
    assert abs(pc[:, 0].mean() - exact) <= 4 * pc[:, 0].std() + 1e-6 * abs(exact)
    assert abs(pc[:, 1].mean() - exact_dl) <= 4 * pc[:, 1].std() + 1e-6 * abs(exact_dl)


def test_nlml_afn_rejects_bad_arguments(agp):
    X, _ = points(300, 4, 16, np.float64)
    W = [[0, 1], [2, 3]]
    plan = make(agp, X, W, np.float64, "gauss", (0.2, 1.0, 0.1))
    afn = plan.afn(10, 5)
    y = torch.ones(300, dtype=torch.float64, device=DEV)
    with pytest.raises(agp.AgpError):
        afn.nlml_grad(y, torch.ones(300, 32, dtype=torch.float64, device=DEV))
    plan.set_hyper(0.3, 1.0, 0.1)
    with pytest.raises(agp.AgpError):
        afn.nlml_grad(y, torch.ones(300, 4, dtype=torch.float64, device=DEV))
