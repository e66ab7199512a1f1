"""GPU parity of the solver layer (Sec. 1): batched CG with FP64 scalars, the
SLQ/Hutchinson NLML gradient estimate, and the autograd Function, against the
FP64 CPU oracle on the Fourier-truncated operator."""
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


def o2_matrix(X, W, kind, ell, sf, se, N, which=None, block=128):
    """The Fourier-truncated operator (or a derivative operator) as a dense
    matrix, built column block by column block from the oracle."""
    n = X.shape[0]
    M = np.zeros((n, n))
    for a in range(0, n, block):
        E = np.zeros((n, min(block, n - a)))
        E[np.arange(a, a + E.shape[1]), np.arange(E.shape[1])] = 1.0
        if which is None:
            M[:, a:a + E.shape[1]] = O.truncated_matvec(X, W, kind, ell, sf, se, E, N)
        else:
            M[:, a:a + E.shape[1]] = O.truncated_deriv_matvec(X, W, kind, ell, sf, se, E, N, which)
    return 0.5 * (M + M.T)


def small_problem(n=1500, seed=21, dtype=np.float64):
    rng = np.random.default_rng(seed)
    X = inputs.to_precision(inputs.minmax_scale(rng.standard_normal((n, 4))), dtype).astype(np.float64)
    return X, [[0, 1], [2, 3]], rng


# ---------------------------------------------------------------------------
# CG
# ---------------------------------------------------------------------------
def test_cg_fp64_matches_dense_solve(agp):
    X, W, rng = small_problem()
    th = dict(kind="gauss", ell=0.3, sf=1.0, se=0.3)
    K = o2_matrix(X, W, th["kind"], th["ell"], th["sf"], th["se"], 32)
    B = rng.standard_normal((X.shape[0], 4))
    plan = agp.Plan(torch.tensor(X, device=DEV), W, 32, 5, th["kind"], th["ell"], th["sf"], th["se"])
    Xs, it, relres = plan.solve(torch.tensor(B, device=DEV), rtol=1e-10, maxit=1000)
    ref = np.linalg.solve(K, B)
    assert rel(Xs.cpu().numpy(), ref) <= 1e-7
    assert np.all(relres <= 1e-10)
    _, it_o, _, _, _ = O.cg(lambda P: K @ P, B, rtol=1e-10, maxit=1000)
    # rounding paths differ (operator within 1e-8, summation order): counts agree loosely
    assert np.all(it <= 1.25 * it_o), (it, it_o)


def test_cg_fp32_true_residual_and_not_converged(agp):
    X, W, rng = small_problem(dtype=np.float32)
    K = o2_matrix(X, W, "matern12", 0.4, 1.0, 0.2, 32)
    B = rng.standard_normal((X.shape[0], 5))
    plan = agp.Plan(torch.tensor(X, dtype=torch.float32, device=DEV), W, 32, 5, "matern12", 0.4,
                    1.0, 0.2)
    Bt = torch.tensor(B, dtype=torch.float32, device=DEV)
    # kappa(K) ~ 7e4: residuals recomputed from FP32 matvecs (residual
    # replacement) carry noise near 1e-4 here (measured: columns stop at
    # 4e-5 .. 9.95e-5 after 220-345 steps, and an occasional column cannot
    # certify 1e-4 at all), so the test asks for 3e-4
    Xs, it, relres = plan.solve(Bt, rtol=3e-4, maxit=3000)
    Xn = Xs.cpu().numpy().astype(np.float64)
    true = np.linalg.norm(B - K @ Xn, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(relres <= 3e-4)
    # CG converged on the FP32 operator K~ = K + E, |E| <= e_mv |K|; then
    # |b - K x| <= rtol |b| + e_mv |K| |x|: the true residual may exceed rtol
    # by the FP32 matvec error amplified by the solution norm.
    KX = plan.matvec(Xs).cpu().numpy().astype(np.float64)
    e_mv = np.linalg.norm(KX - K @ Xn, axis=0) / np.linalg.norm(K @ Xn, axis=0)
    bound = 3e-4 + 2 * e_mv * np.linalg.norm(K @ Xn, axis=0) / np.linalg.norm(B, axis=0) \
        * np.linalg.norm(K, 2) * np.linalg.norm(Xn, axis=0) / np.linalg.norm(K @ Xn, axis=0)
    assert np.all(true <= bound), (true, bound)
    with pytest.raises(agp.AgpError) as ei:
        plan.solve(Bt, rtol=1e-12, maxit=3)
    assert ei.value.status == agp.AGP_NOT_CONVERGED
    _, it, relres = plan.solve(Bt, rtol=1e-12, maxit=3, raise_not_converged=False)
    assert np.all(it == 3) and np.all(relres > 1e-12)


def test_cg_batched_pcg_workload_subset_fp64(agp):
    # Matern(1/2), four d=3 windows, [y, 3 probes]. Unpreconditioned, the
    # condition number here is ~1e6 (sigma_eps^2 = 0.0025): FP32 CG stalls
    # above the 1e-4 target, which is why the paper preconditions. With FP64
    # matvecs plain CG reaches 1e-4 within the iteration cap.
    w = inputs.subset(inputs.batched_pcg(n=3000, R=4), 3000)
    plan = agp.Plan(torch.tensor(w.X, device=DEV), w.windows, w.N, w.cutoff, w.kernel, w.ell,
                    w.sigma_f, w.sigma_eps)
    Xs, it, relres = plan.solve(torch.tensor(w.V, device=DEV), rtol=1e-4, maxit=3000)
    Xn = Xs.cpu().numpy()
    KX = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, Xn, w.N)
    true = np.linalg.norm(w.V - KX, axis=0) / np.linalg.norm(w.V, axis=0)
    assert np.all(relres <= 1e-4)
    assert np.all(true <= 2e-4), true


# ---------------------------------------------------------------------------
# NLML gradient (SLQ + Hutchinson, M = I)
# ---------------------------------------------------------------------------
def test_nlml_exact_with_orthogonal_probes_fp64(agp):
    # n probes sqrt(n) q_i from an orthogonal basis and n Lanczos steps make the
    # estimator exact: it must return the exact NLML of the truncated operator
    # and its exact gradient.
    n = 48
    X, W, rng = small_problem(n, seed=5)
    th = dict(kind="gauss", ell=0.25, sf=0.9, se=0.5)
    K = o2_matrix(X, W, th["kind"], th["ell"], th["sf"], th["se"], 16)
    y = rng.standard_normal(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Z = math.sqrt(n) * Q
    plan = agp.Plan(torch.tensor(X, device=DEV), W, 16, 5, th["kind"], th["ell"], th["sf"], th["se"])
    nl, g = plan.nlml_grad(torch.tensor(y, device=DEV), torch.tensor(Z, device=DEV),
                           lanczos_steps=n)
    assert nl == pytest.approx(O.nlml_exact(K, y), rel=1e-7)
    Ki = np.linalg.inv(K)
    a = Ki @ y
    for which in ["ell", "sigma_f", "sigma_eps"]:
        dK = o2_matrix(X, W, th["kind"], th["ell"], th["sf"], th["se"], 16, which)
        exact = 0.5 * (-(a @ dK @ a) + np.trace(Ki @ dK))
        assert g[which] == pytest.approx(exact, rel=1e-6, abs=1e-8), which


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-7), (torch.float32, 2e-3)])
def test_nlml_matches_oracle_estimator(agp, dtype, tol):
    # Same probes, same 20 steps: the GPU estimator against the oracle's.
    npdt = np.float32 if dtype == torch.float32 else np.float64
    X, W, rng = small_problem(1200, seed=8, dtype=npdt)
    th = dict(kind="gauss", ell=math.log(2), sf=math.log(2), se=math.log(2))
    K = o2_matrix(X, W, th["kind"], th["ell"], th["sf"], th["se"], 32)
    dK = {w: o2_matrix(X, W, th["kind"], th["ell"], th["sf"], th["se"], 32, w)
          for w in ["ell", "sigma_f", "sigma_eps"]}
    y = rng.standard_normal(1200)
    Z = inputs.rademacher(1200, 16, 99)
    nl_o, g_o = O.nlml_estimate(lambda P: K @ P, {w: (lambda P, M=M: M @ P) for w, M in dK.items()},
                                y, Z, lanczos_steps=20, rtol=0, maxit=20)
    # the oracle's y-solve above runs to rtol=0 within 20 steps, like the GPU's
    plan = agp.Plan(torch.tensor(X, dtype=dtype, device=DEV), W, 32, 5, th["kind"], th["ell"],
                    th["sf"], th["se"])
    nl, g = plan.nlml_grad(torch.tensor(y, dtype=dtype, device=DEV),
                           torch.tensor(Z, dtype=dtype, device=DEV), lanczos_steps=20)
    assert nl == pytest.approx(nl_o, rel=tol)
    for k in g:
        assert g[k] == pytest.approx(g_o[k], rel=10 * tol, abs=10 * tol * abs(nl_o) / 1200), k


# ---------------------------------------------------------------------------
# autograd Function
# ---------------------------------------------------------------------------
def test_autograd_gradcheck_fp64(agp):
    from paper_2504_00480_gb300.autograd import additive_kernel_matvec
    X, W, rng = small_problem(60, seed=3)
    plan = agp.Plan(torch.tensor(X, device=DEV), W, 16, 4, "matern12", 0.3, 1.0, 0.2)
    V = torch.tensor(rng.standard_normal((60, 2)), device=DEV, requires_grad=True)
    th = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (0.3, 1.1, 0.2)]
    f = lambda V, a, b, c: additive_kernel_matvec(plan, V, a, b, c)
    # FP64 atomics reorder additions between calls: allow rounding-level nondeterminism
    assert torch.autograd.gradcheck(f, (V, *th), eps=1e-6, atol=1e-7, rtol=1e-5, nondet_tol=1e-10)


def test_autograd_autograd_workload_vs_fd_and_oracles(agp):
    # Autograd workload shape (three d=3 windows, Gaussian ell=0.2, sigma_f=1,
    # sigma_eps=0.1, N=32, s=5) on its first 5,000 points, FP64 plan:
    # L = sum(W * K_hat V).
    from paper_2504_00480_gb300.autograd import additive_kernel_matvec
    w = inputs.subset(inputs.autograd(n=5000, R=1), 5000)
    Wt = w.extra["W"]
    plan = agp.Plan(torch.tensor(w.X, device=DEV), w.windows, w.N, w.cutoff, w.kernel, w.ell,
                    w.sigma_f, w.sigma_eps)
    V = torch.tensor(w.V, device=DEV, requires_grad=True)
    th = [torch.tensor(v, dtype=torch.float64, requires_grad=True)
          for v in (w.ell, w.sigma_f, w.sigma_eps)]
    Wd = torch.tensor(Wt, device=DEV)
    L = (Wd * additive_kernel_matvec(plan, V, *th)).sum()
    gV, ge, gf, gs = torch.autograd.grad(L, [V] + th)
    # dL/dV = K_hat W (symmetric operator) against the truncated-sum oracle
    refV = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, Wt, w.N)
    assert rel(gV.cpu().numpy(), refV) <= 1e-5
    # hyperparameter gradients: against the truncated-sum oracle ...
    got = {"ell": float(ge), "sigma_f": float(gf), "sigma_eps": float(gs)}
    for k in got:
        ref = float(np.sum(Wt * O.truncated_deriv_matvec(w.X, w.windows, w.kernel, w.ell,
                                                         w.sigma_f, w.sigma_eps, w.V, w.N, k)))
        assert got[k] == pytest.approx(ref, rel=1e-5), k
        # ... and against the dense oracle's gradient, within the truncation
        # error of the Fourier series at this (ell, N) (no boundary smoothing):
        # on these inputs the truncated sum moves these gradients by 2.7e-4
        # (ell) and 5.5e-5 (sigma_f) relative, so 2e-3 leaves a 7x margin.
        dense = float(np.sum(Wt * O.dense_deriv_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f,
                                                       w.sigma_eps, w.V, k)))
        assert got[k] == pytest.approx(dense, rel=2e-3), k
    # ... and against central finite differences of the GPU operator (h = 1e-4)
    h = 1e-4
    base = dict(ell=w.ell, sigma_f=w.sigma_f, sigma_eps=w.sigma_eps)
    Vt = V.detach()
    for k in got:
        def L_at(x):
            t = dict(base, **{k: x})
            with torch.no_grad():
                return float((Wd * additive_kernel_matvec(plan, Vt, t["ell"], t["sigma_f"],
                                                          t["sigma_eps"])).sum())
        fd = (L_at(base[k] + h) - L_at(base[k] - h)) / (2 * h)
        assert got[k] == pytest.approx(fd, rel=1e-5), k


# ---------------------------------------------------------------------------
# device-drawn Rademacher probes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_rademacher_probes_match_the_oracle_generator(agp, dtype):
    n, R, seed = 100_003, 17, 0xC0FFEE
    Z = agp.agp_rademacher(n, R, seed, dtype=dtype, device=DEV).cpu().numpy()
    np.testing.assert_array_equal(Z, O.rademacher_probes(n, R, seed))


def test_nlml_grad_seed_equals_nlml_grad_with_the_same_probes(agp):
    # 6 CG-Lanczos steps: on this matrix (eigenvalues 0.96 .. 119 and one at
    # 1905) finite-precision CG loses orthogonality after about six steps,
    # and from then on its iterates depend on the rounding sequence, which
    # the order of the FP64 atomic additions changes from run to run
    # (measured run-to-run iterate differences 1e-16, 1e-10, 2e-7, 5e-3
    # after 2, 6, 8, 10 steps; the CPU oracle's CG shows the same growth
    # under a 1e-11 change of the operator)
    X, W, rng = small_problem(n=1200, seed=31)
    plan = agp.Plan(torch.tensor(X, device=DEV), W, 32, 5, "gauss", 0.2, 1.0, 1.0)
    y = torch.tensor(rng.standard_normal(1200), device=DEV)
    seed = 424242
    nl_s, g_s = plan.nlml_grad_seed(y, 12, seed, lanczos_steps=6)
    Z = torch.tensor(O.rademacher_probes(1200, 12, seed), device=DEV)
    nl, g = plan.nlml_grad(y, Z, lanczos_steps=6)
    # the same probes: the two runs differ only by the order of the FP64
    # atomic additions inside the matvecs
    assert nl_s == pytest.approx(nl, rel=1e-9)
    for k in g:
        assert g_s[k] == pytest.approx(g[k], rel=1e-6, abs=1e-9), k
    plan.close()
