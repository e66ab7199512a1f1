"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: relative l2 error <= 1e-5 for the FP64 plan and <= 1e-4 for the
FP32 plan against the Fourier-truncated sum of Sec. 3.1 eq. (3.3) (the
quantity the method computes up to the NFFT window error); bin indices
bit-exact. Sizes span many work items (grid cells) and ragged tails.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_00480_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

TOL = {torch.float64: 1e-5, torch.float32: 1e-4}
DEV = "cuda:0"


@pytest.fixture(scope="module")
def agp():
    from paper_2504_00480_gb300 import agp as A
    from paper_2504_00480_gb300 import build
    build.build()
    A.load_library()
    return A


def rel(a, b):
    """Relative l2 error (complex arrays keep their imaginary parts); an
    all-zero reference requires an all-zero result."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    if nb == 0:
        return 0.0 if np.linalg.norm(a) == 0 else float("inf")
    return float(np.linalg.norm(a - b) / nb)


def make(agp, X, windows, N, s, kernel="gauss", ell=0.3, sf=1.0, se=0.1, dtype=torch.float32):
    Xt = torch.tensor(X, dtype=dtype, device=DEV)
    return agp.Plan(Xt, windows, N, s, kernel, ell, sf, se)


def points(rng, n, p, dtype=np.float32, gauss=False):
    raw = rng.standard_normal((n, p)) if gauss else rng.uniform(-1, 1, (n, p))
    return inputs.to_precision(inputs.minmax_scale(raw), dtype).astype(np.float64)


# ---------------------------------------------------------------------------
# a0: bins, bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("N", [8, 32, 64])
def test_bins_bit_exact(agp, dtype, N):
    rng = np.random.default_rng(100 + N)
    npdt = np.float32 if dtype == torch.float32 else np.float64
    X = rng.uniform(-0.25, 0.25, size=(5000, 6)).astype(npdt)
    # coordinates on and next to cell boundaries
    n_os = 2 * N
    edges = (np.arange(-N // 2, N // 2) / n_os).astype(npdt)
    X[:len(edges), 0] = edges
    X[len(edges):2 * len(edges), 1] = np.nextafter(edges, npdt(-1))[::-1].clip(-0.25, None)
    X[:3, 2] = [-0.25, np.nextafter(npdt(0.25), npdt(0)), 0.0]
    X = X.astype(np.float64)
    W = [[0, 1, 2], [3, 4], [5]]
    plan = make(agp, X, W, N, 2, dtype=dtype)
    for s, w in enumerate(W):
        got = plan.bins(s).cpu().numpy()
        want = O.bins(X[:, w], n_os)
        np.testing.assert_array_equal(got, want)


def test_domain_error(agp):
    X = np.zeros((10, 2))
    X[3, 1] = 0.25                      # outside [-1/4, 1/4)
    with pytest.raises(agp.AgpError) as ei:
        make(agp, X, [[0, 1]], 32, 4)
    assert ei.value.status == agp.AGP_EDOMAIN


# ---------------------------------------------------------------------------
# a1: coefficients b_k (FP64 on the device)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["gauss", "matern12", "matern32", "imq", "sinc"])
@pytest.mark.parametrize("d,N", [(1, 32), (2, 64), (3, 32), (3, 16)])
def test_coeffs_match_oracle(agp, kind, d, N):
    rng = np.random.default_rng(7)
    X = points(rng, 50, d)
    plan = make(agp, X, [list(range(d))], N, 4, kind, ell=0.23, dtype=torch.float64)
    for der in (False, True):
        got = plan.coeffs(0, der)
        want = O.fourier_coeffs(kind, 0.23, N, d, der).real
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    plan.set_hyper(0.41, 1.0, 0.1)
    want = O.fourier_coeffs(kind, 0.41, N, d).real
    assert np.max(np.abs(plan.coeffs(0) - want)) <= 1e-13 * np.max(np.abs(want))


# ---------------------------------------------------------------------------
# NFFT halves against the exact NDFT
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("d,N,s,n", [(1, 16, 5, 900), (2, 32, 5, 3000), (3, 16, 5, 2500),
                                     (3, 32, 6, 1500), (2, 64, 5, 2000)])
def test_adjoint_nfft_vs_ndft(agp, dtype, d, N, s, n):
    rng = np.random.default_rng(d * 100 + N + s)
    X = points(rng, n, d, np.float32 if dtype == torch.float32 else np.float64, gauss=True)
    V = rng.standard_normal((n, 3))
    plan = make(agp, X, [list(range(d))], N, s, dtype=dtype)
    got = plan.adjoint_nfft(0, torch.tensor(V, dtype=dtype, device=DEV)).cpu().numpy()
    want = np.moveaxis(O.ndft_adjoint(X, V, N), -1, 0)
    assert rel(got, want) <= (1e-7 if dtype == torch.float64 else 1e-5)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("d,N,s,n", [(1, 16, 5, 700), (2, 32, 5, 2500), (3, 16, 5, 2000),
                                     (3, 32, 4, 1200)])
def test_nfft_real_vs_ndft(agp, dtype, d, N, s, n):
    rng = np.random.default_rng(d * 10 + N + s)
    X = points(rng, n, d, np.float32 if dtype == torch.float32 else np.float64)
    R = 2
    F = rng.standard_normal((N,) * d + (R,)) + 1j * rng.standard_normal((N,) * d + (R,))
    plan = make(agp, X, [list(range(d))], N, s, dtype=dtype)
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    fh = torch.tensor(np.moveaxis(F, -1, 0).copy(), dtype=cdt, device=DEV)
    got = plan.nfft_real(0, fh).cpu().numpy()
    want = np.real(O.ndft(X, F, N))
    tol = 1e-4 if s == 4 and dtype == torch.float64 else (1e-7 if dtype == torch.float64 else 1e-5)
    assert rel(got, want) <= tol


# ---------------------------------------------------------------------------
# Matvec and derivative matvecs against the truncated sum (O2)
# ---------------------------------------------------------------------------
def check_matvec(agp, w, dtype, R=None, rows=None):
    V = w.V if R is None else w.V[:, :R]
    plan = make(agp, w.X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps, dtype)
    Vt = torch.tensor(V, dtype=dtype, device=DEV)
    got = plan.matvec(Vt).cpu().numpy()
    want = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, V, w.N)
    e = rel(got, want)
    assert e <= TOL[dtype], e
    for which in ["ell", "sigma_f", "sigma_eps"]:
        got = plan.deriv_matvec(which, Vt).cpu().numpy()
        want = O.truncated_deriv_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f,
                                        w.sigma_eps, V, w.N, which)
        e = rel(got, want)
        assert e <= TOL[dtype], (which, e)
    return plan


def test_plain_fp64_full_config(agp):
    # n=1000, d=2, Gaussian ell=0.3, N=32, s=4, FP64, one RHS.
    w = inputs.plain_fp64()
    plan = check_matvec(agp, w, torch.float64)
    # Against the dense sum the error is O2's own truncation error (no
    # boundary smoothing, Sec. 3.1): the GPU reproduces it.
    Vt = torch.tensor(w.V, dtype=torch.float64, device=DEV)
    got = plan.matvec(Vt).cpu().numpy()
    dense = O.dense_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, w.V)
    trunc = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, w.V, w.N)
    assert abs(rel(got, dense) - rel(trunc, dense)) <= 1e-5


def test_dense_oracle_small_lengthscale_fp64(agp):
    # Small ell: truncation is negligible, so the GPU meets the dense sum itself.
    rng = np.random.default_rng(3)
    X = points(rng, 2000, 3, np.float64)
    V = rng.standard_normal((2000, 2))
    plan = make(agp, X, [[0, 1], [2]], [64, 64], 6, "gauss", 0.03, 1.0, 0.1, torch.float64)
    got = plan.matvec(torch.tensor(V, device=DEV)).cpu().numpy()
    dense = O.dense_matvec(X, [[0, 1], [2]], "gauss", 0.03, 1.0, 0.1, V)
    assert rel(got, dense) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_autograd_workload_subset(agp, dtype):
    w = inputs.subset(inputs.autograd(n=4000, R=3), 4000)
    check_matvec(agp, w, dtype)


@pytest.mark.parametrize("R", [1, 5, 32])
def test_batched_pcg_workload_subset_matern(agp, R):
    w = inputs.subset(inputs.batched_pcg(n=3000), 3000)
    check_matvec(agp, w, torch.float32, R=R)


@pytest.mark.parametrize("R", [12, 17, 24, 32, 40])
def test_nlml_workload_subset_mixed_d(agp, R):
    w = inputs.subset(inputs.nlml_grad(n=3000, R=40), 3000)
    check_matvec(agp, w, torch.float32, R=R)


def test_uneven_problem_s4(agp):
    w = inputs.uneven_batch(n_problems=1, n_lo=3000, n_hi=3001)[0]
    check_matvec(agp, w, torch.float32)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_single_point_and_single_cell(agp, dtype):
    X = np.array([[0.01, -0.2, 0.24]])
    V = np.array([[1.5, -2.0]])
    plan = make(agp, X, [[0, 1, 2]], 32, 5, dtype=dtype)
    got = plan.matvec(torch.tensor(V, dtype=dtype, device=DEV)).cpu().numpy()
    want = O.truncated_matvec(X, [[0, 1, 2]], "gauss", 0.3, 1.0, 0.1, V, 32)
    assert rel(got, want) <= TOL[dtype]
    # 700 points in one cell: several work items of one cell
    rng = np.random.default_rng(5)
    X = 6.0 / 64 + rng.uniform(0, 1.0 / 64, size=(700, 3)) * 0.999   # cell 6 of n_os = 64
    V = rng.standard_normal((700, 3))
    plan = make(agp, X, [[0, 1, 2]], 32, 5, dtype=dtype)
    assert plan.query(0)["n_items"] == math.ceil(700 / 256)
    got = plan.matvec(torch.tensor(V, dtype=dtype, device=DEV)).cpu().numpy()
    want = O.truncated_matvec(X, [[0, 1, 2]], "gauss", 0.3, 1.0, 0.1, V, 32)
    assert rel(got, want) <= TOL[dtype]


@pytest.mark.parametrize("s,N", [(2, 8), (3, 16), (6, 32), (5, 64)])
def test_cutoffs_and_bandwidths(agp, s, N):
    rng = np.random.default_rng(s * N)
    X = points(rng, 1500, 4, np.float64)
    V = rng.standard_normal((1500, 2))
    W = [[0, 1, 2], [3]]
    plan = make(agp, X, W, N, s, "matern12", 0.2, 0.9, 0.3, torch.float64)
    got = plan.matvec(torch.tensor(V, device=DEV)).cpu().numpy()
    want = O.truncated_matvec(X, W, "matern12", 0.2, 0.9, 0.3, V, N)
    # the NFFT window error falls like exp(-2 pi s sqrt(1/2)): s=2 is coarse
    assert rel(got, want) <= {2: 5e-3, 3: 2e-4}.get(s, 1e-5)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind", ["matern32", "imq", "sinc"])
def test_further_kernels_matvec_and_derivatives(agp, dtype, kind):
    # the kernels of Sec. 4 beyond eq. (2.2) on mixed windows (d = 3, 2, 1)
    rng = np.random.default_rng(32)
    npdt = np.float32 if dtype == torch.float32 else np.float64
    X = points(rng, 2500, 6, npdt)
    W = [[0, 1, 2], [3, 4], [5]]
    w = inputs.Workload(kind, X, W, kind, 0.2, 0.8, 0.3, [32, 32, 32], 5, npdt,
                        V=rng.standard_normal((2500, 9)))
    check_matvec(agp, w, dtype)


def test_strided_blocks_and_noise_flag(agp):
    rng = np.random.default_rng(9)
    X = points(rng, 2000, 3)
    V = rng.standard_normal((2000, 12))
    plan = make(agp, X, [[0, 1, 2]], 32, 5, ell=0.25, sf=1.2, se=0.3)
    Vt = torch.tensor(V, dtype=torch.float32, device=DEV)
    big = torch.zeros((2000, 20), dtype=torch.float32, device=DEV)
    out = big[:, 3:10]                      # ldo = 20, R = 7, unaligned
    agp_mod = agp
    agp_mod.agp_matvec(plan.handle, Vt[:, 2:9], out, add_noise=False)
    got = out.cpu().numpy()
    want = O.truncated_matvec(X, [[0, 1, 2]], "gauss", 0.25, 1.2, 0.3, V[:, 2:9], 32,
                              add_noise=False)
    assert rel(got, want) <= 1e-4
    assert float(big[:, :3].abs().max()) == 0.0 and float(big[:, 10:].abs().max()) == 0.0


def test_out_overlapping_v_rejected(agp):
    rng = np.random.default_rng(1)
    X = points(rng, 100, 2)
    plan = make(agp, X, [[0, 1]], 16, 4)
    V = torch.zeros((100, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(agp.AgpError) as ei:
        agp.agp_matvec(plan.handle, V, V)
    assert ei.value.status == agp.AGP_EINVAL


def test_symmetry_fp64(agp):
    rng = np.random.default_rng(11)
    X = points(rng, 3000, 5, np.float64, gauss=True)
    W = [[0, 1, 2], [3, 4]]
    plan = make(agp, X, W, [32, 64], 5, "matern12", 0.3, 1.0, 0.2, torch.float64)
    v = torch.tensor(rng.standard_normal((3000, 1)), device=DEV)
    u = torch.tensor(rng.standard_normal((3000, 1)), device=DEV)
    a = float((u * plan.matvec(v)).sum())
    b = float((v * plan.matvec(u)).sum())
    assert abs(a - b) <= 1e-11 * abs(a)


# ---------------------------------------------------------------------------
# Full size, in the launch configuration the benchmark times: n = 1,000,000,
# windows d = (3, 3, 2), N = (32, 32, 64), s = 5, 32 right-hand sides, FP32.
# Checked on sampled outputs the oracle computes one by one.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def full(agp):
    w = inputs.nlml_grad()
    plan = make(agp, w.X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    return w, plan


def test_full_size_bins_bit_exact(full):
    w, plan = full
    for s, win in enumerate(w.windows):
        got = plan.bins(s).cpu().numpy()
        np.testing.assert_array_equal(got, O.bins(w.X[:, win], 2 * w.N[s]))


def test_full_size_adjoint_nfft_sampled_frequencies(full):
    # c_k = sum_j v_j exp(-2 pi i k.x_j) for 40 sampled k, all 32 columns.
    w, plan = full
    rng = np.random.default_rng(0)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    for s, win in enumerate(w.windows):
        N, d = w.N[s], len(win)
        chat = plan.adjoint_nfft(s, V).cpu().numpy()          # [R][N]*d
        ks = rng.integers(-N // 2, N // 2, size=(40, d))
        x = w.X[:, win]
        got = np.stack([chat[(slice(None),) + tuple(k + N // 2)] for k in ks])   # [40][R]
        ph = np.exp(-2j * np.pi * (x @ ks.T))                   # [n][40]
        want = ph.T @ w.V                                        # [40][R]
        assert rel(got, want) <= 1e-5


def test_full_size_matvec_sampled_rows(full):
    # One column through the full matvec, 64 sampled output rows against O2
    # (c_k of every window over all n points, then the outer sum per row).
    w, plan = full
    rng = np.random.default_rng(1)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    out = plan.matvec(V).cpu().numpy()
    rows = np.sort(rng.choice(w.n, size=64, replace=False))
    want = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                              w.V[:, :1], w.N, rows=rows)
    assert rel(out[rows, :1], want) <= 1e-4
