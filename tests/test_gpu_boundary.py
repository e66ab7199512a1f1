"""GPU parity of the outer boundary smoothing of kappa_R (Sec. 3.1) through
the C ABI (agp_plan_set_boundary) against the FP64 oracle.

Coefficients: the device builds the boundary polynomial from Taylor jets
and a p x p solve, the oracle from Cauchy-integral derivatives and the full
2p x 2p system; both then sample and transform in FP64, so they agree to
1e-10 of the largest coefficient. Matvecs: relative l2 error <= 1e-5 (FP64
plan) and <= 1e-4 (FP32 plan) against the smoothed truncated sum, as for the
unsmoothed operator.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_00480_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

TOL = {torch.float64: 1e-5, torch.float32: 1e-4}
DEV = "cuda:0"
KINDS = ["gauss", "matern12", "matern32", "imq", "sinc"]


@pytest.fixture(scope="module")
def agp():
    from paper_2504_00480_gb300 import agp as A
    from paper_2504_00480_gb300 import build
    build.build()
    A.load_library()
    return A


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def ball_points(rng, n, p, windows, eps_b, npdt):
    """Standard normal features, min-max scaled, each window scaled into the
    ball of radius 1/4 - eps_b/2 (with a margin for the rounding to npdt)."""
    X = inputs.minmax_scale(rng.standard_normal((n, p)))
    X = inputs.ball_scale(X, windows, 0.999 * (0.25 - eps_b / 2))
    return inputs.to_precision(X, npdt).astype(np.float64)


def make(agp, X, windows, N, s, kernel, ell, sf=1.0, se=0.1, dtype=torch.float64):
    Xt = torch.tensor(X, dtype=dtype, device=DEV)
    return agp.Plan(Xt, windows, N, s, kernel, ell, sf, se)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d,N", [(1, 32), (2, 64), (3, 16), (3, 32)])
@pytest.mark.parametrize("eps_b,p", [(0.125, 4), (0.0625, 2), (0.1875, 8)])
def test_coeffs_match_oracle(agp, kind, d, N, eps_b, p):
    rng = np.random.default_rng(11)
    W = [list(range(d))]
    X = ball_points(rng, 60, d, W, eps_b, np.float64)
    plan = make(agp, X, W, N, 4, kind, ell=0.23)
    plain = plan.coeffs(0).copy()
    plan.set_boundary(eps_b, p)
    for der in (False, True):
        got = plan.coeffs(0, der)
        want = O.fourier_coeffs(kind, 0.23, N, d, der, boundary=(eps_b, p)).real
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want)), der
    # a new ell keeps the smoothing
    plan.set_hyper(0.41, 1.0, 0.1)
    want = O.fourier_coeffs(kind, 0.41, N, d, boundary=(eps_b, p)).real
    assert np.max(np.abs(plan.coeffs(0) - want)) <= 1e-10 * np.max(np.abs(want))
    # switched off: the plain coefficients again, bit for bit
    plan.set_hyper(0.23, 1.0, 0.1)
    plan.set_boundary(0.0, 0)
    np.testing.assert_array_equal(plan.coeffs(0), plain)


@pytest.mark.parametrize("dtype,R", [(torch.float64, 3), (torch.float32, 9), (torch.float32, 20)])
@pytest.mark.parametrize("kind", ["gauss", "matern32", "sinc"])
def test_matvec_and_derivatives_match_oracle(agp, dtype, R, kind):
    """Mixed windows (d = 3, 2, 1); FP32 with 9 and 20 columns takes the
    tensor-core passes of both grid widths on the d = 3 window."""
    rng = np.random.default_rng(21)
    npdt = np.float32 if dtype == torch.float32 else np.float64
    W = [[0, 1, 2], [3, 4], [5]]
    eps_b, p = 0.125, 4
    X = ball_points(rng, 2400, 6, W, eps_b, npdt)
    V = rng.standard_normal((2400, R))
    Ns = [32, 32, 32]
    plan = make(agp, X, W, Ns, 5, kind, 0.25, 0.8, 0.3, dtype)
    plan.set_boundary(eps_b, p)
    Vt = torch.tensor(V, dtype=dtype, device=DEV)
    b = (eps_b, p)
    got = plan.matvec(Vt).cpu().numpy()
    want = O.truncated_matvec(X, W, kind, 0.25, 0.8, 0.3, V, Ns, boundary=b)
    assert rel(got, want) <= TOL[dtype]
    for which in ("ell", "sigma_f"):
        got = plan.deriv_matvec(which, Vt).cpu().numpy()
        want = O.truncated_deriv_matvec(X, W, kind, 0.25, 0.8, 0.3, V, Ns, which, boundary=b)
        assert rel(got, want) <= TOL[dtype], which
    plan.check()


def test_smoothing_brings_the_gpu_sum_closer_to_the_dense_sum(agp):
    """Gaussian ell = 0.3 on one d = 3 window, N = 32, s = 5, FP64: the
    smoothed operator is several times closer to the dense kernel sum."""
    rng = np.random.default_rng(5)
    W = [[0, 1, 2]]
    eps_b, p = 0.125, 4
    X = ball_points(rng, 3000, 3, W, eps_b, np.float64)
    V = rng.standard_normal((3000, 1))
    plan = make(agp, X, W, 32, 5, "gauss", 0.3, 1.0, 0.0)
    Vt = torch.tensor(V, dtype=torch.float64, device=DEV)
    rows = np.arange(0, 3000, 7)
    dense = O.dense_matvec(X, W, "gauss", 0.3, 1.0, 0.0, V, rows=rows)
    e_plain = rel(plan.matvec(Vt).cpu().numpy()[rows], dense)
    plan.set_boundary(eps_b, p)
    e_smooth = rel(plan.matvec(Vt).cpu().numpy()[rows], dense)
    assert e_smooth < e_plain / 5, (e_plain, e_smooth)


def test_points_outside_the_ball_are_rejected(agp):
    rng = np.random.default_rng(9)
    W = [[0, 1, 2], [3, 4]]
    X = inputs.minmax_scale(rng.standard_normal((500, 5)))    # box, not ball
    plan = make(agp, X, W, 16, 4, "gauss", 0.3)
    before = [plan.coeffs(0).copy(), plan.coeffs(1).copy()]
    with pytest.raises(agp.AgpError) as ei:
        plan.set_boundary(0.125, 4)
    assert ei.value.status == agp.AGP_EDOMAIN
    np.testing.assert_array_equal(plan.coeffs(0), before[0])
    np.testing.assert_array_equal(plan.coeffs(1), before[1])
    for eps_b, p in ((-0.1, 4), (0.3, 4), (0.125, 9), (0.125, -1)):
        with pytest.raises(agp.AgpError) as ei:
            plan.set_boundary(eps_b, p)
        assert ei.value.status == agp.AGP_EINVAL
    # the plan is still usable
    V = torch.ones((500, 2), dtype=torch.float64, device=DEV)
    out = plan.matvec(V).cpu().numpy()
    want = O.truncated_matvec(X, W, "gauss", 0.3, 1.0, 0.1, np.ones((500, 2)), 16)
    assert rel(out, want) <= 1e-4     # s = 4 window error
