"""Spreading and interpolation on the tensor cores (tcgen05, split TF32):
the matvec and the derivative operators with each tensor-core kernel
family (3, the default: both persistent kernels with A in tensor memory; 1:
tensor-memory spreading, shared-memory interpolation; 2: both with operands
in shared memory) against the oracle at the FP32 tolerance, against the
FMA-pipe kernels of the same plan, for both supported cutoffs, a ragged right-hand-side count,
strided blocks and the full-size workload on sampled rows. 17 .. 32
right-hand sides run in passes of 32 grid columns, 9 .. 16 in passes of 16."""
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


def points(rng, n, p):
    X = inputs.minmax_scale(rng.standard_normal((n, p)))
    return inputs.to_precision(X, np.float32).astype(np.float64)


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("s,N,R", [(5, 32, 32), (5, 32, 17), (4, 16, 32), (5, 16, 25),
                                   (5, 32, 12), (4, 16, 9)])
def test_tc_spread_matches_oracle_and_fma_path(agp, s, N, R, mode):
    rng = np.random.default_rng(100 + s + R)
    n = 4000
    X = points(rng, n, 7)
    W = [[0, 1, 2], [3, 4, 5], [6]]
    V = rng.standard_normal((n, R))
    plan = agp.Plan(torch.tensor(X, dtype=torch.float32, device=DEV), W, N, s, "gauss",
                    0.15, 0.9, 0.2)
    Vt = torch.tensor(V, dtype=torch.float32, device=DEV)
    plan.set_tensor_cores(False)
    ref = plan.matvec(Vt).cpu().numpy()
    plan.set_tensor_cores(mode)
    # the kernels that run (rows of R values: 16-byte aligned only when R % 4
    # == 0, which the persistent spreading kernel stages either way)
    assert plan.kernel_families(R) == (3 if mode in (1, 3) else 2, 3 if mode == 3 else 2)
    got = plan.matvec(Vt).cpu().numpy()
    plan.check()
    want = O.truncated_matvec(X, W, "gauss", 0.15, 0.9, 0.2, V, N)
    assert rel(got, want) <= 1e-4
    assert rel(got, ref) <= 1e-5
    for which in ["ell", "sigma_f", "sigma_eps"]:
        g = plan.deriv_matvec(which, Vt).cpu().numpy()
        wd = O.truncated_deriv_matvec(X, W, "gauss", 0.15, 0.9, 0.2, V, N, which)
        assert rel(g, wd) <= 1e-4, which
    plan.check()


def test_tc_spread_strided_and_adjoint_nfft(agp):
    rng = np.random.default_rng(7)
    n = 3000
    X = points(rng, n, 3)
    V = rng.standard_normal((n, 40))
    plan = agp.Plan(torch.tensor(X, dtype=torch.float32, device=DEV), [[0, 1, 2]], 32, 5,
                    "matern12", 0.2, 1.0, 0.1)
    plan.set_tensor_cores(1)
    Vt = torch.tensor(V, dtype=torch.float32, device=DEV)[:, 3:35]   # ldv = 40, unaligned start
    got = plan.matvec(Vt).cpu().numpy()
    want = O.truncated_matvec(X, [[0, 1, 2]], "matern12", 0.2, 1.0, 0.1, V[:, 3:35], 32)
    assert rel(got, want) <= 1e-4
    V32 = torch.tensor(V[:, :32], dtype=torch.float32, device=DEV)
    c_tc = plan.adjoint_nfft(0, V32).cpu().numpy()
    plan.set_tensor_cores(False)
    c_fma = plan.adjoint_nfft(0, V32).cpu().numpy()
    assert rel(c_tc, c_fma) <= 1e-5
    plan.check()


def test_tc_spread_full_size_sampled_rows(agp):
    w = inputs.nlml_grad(R=32)
    X = torch.tensor(w.X, dtype=torch.float32, device=DEV)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    plan = agp.Plan(X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    plan.set_tensor_cores(False)
    ref = plan.matvec(V)
    plan.set_tensor_cores(True)
    got = plan.matvec(V)
    plan.check()
    assert float((got - ref).norm() / ref.norm()) <= 1e-5
    rows = np.random.default_rng(3).choice(w.X.shape[0], 16, replace=False)
    want = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                              w.V[:, :1], w.N, rows=rows)
    assert rel(got[rows, :1].cpu().numpy(), want) <= 1e-4


def test_tc_full_size_every_operator_sampled_rows(agp):
    """The benchmarked launch configuration (n = 1,000,000, windows d = 3, 3,
    2, 32 right-hand sides in one 32-column pass, tensor-core kernels):
    K_hat and the three derivative operators on 8 columns (both 16-column
    halves of the grid) x 256 sampled rows against the oracle's truncated
    sums over all n points."""
    w = inputs.nlml_grad(R=32)
    X = torch.tensor(w.X, dtype=torch.float32, device=DEV)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    plan = agp.Plan(X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    cols = [0, 3, 7, 12, 17, 22, 26, 31]
    rows = np.sort(np.random.default_rng(5).choice(w.X.shape[0], 256, replace=False))
    want = O.truncated_operators(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                                 w.V[:, cols].astype(np.float32).astype(np.float64), w.N,
                                 rows=rows)
    assert plan.tensor_cores() == 3 and plan.kernel_families(32) == (3, 3)
    for mode in [3, 1, 2]:                   # the default family first
        plan.set_tensor_cores(mode)
        got = {"K": plan.matvec(V)}
        for which in ["ell", "sigma_f", "sigma_eps"]:
            got[which] = plan.deriv_matvec(which, V)
        plan.check()
        for which, g in got.items():
            gs = g[rows][:, cols].double().cpu().numpy()
            for j in range(len(cols)):
                assert rel(gs[:, j], want[which][:, j]) <= 1e-4, (mode, which, cols[j])
    plan.close()
