"""The three-launch DFT stage (forward pruned DFT, spectral multiply, inverse;
Appendix A steps 2 and 4 around Sec. 3.1 eq. (3.3)) that plans and batches
use for their d = 2 and d = 3 windows.

  * FP64: the plan's matvec and ell-derivative matvec equal the oracle's CPU
    NFFT fast sum (adjoint NFFT, coefficients, NFFT; the same window and
    cutoff) to rounding, for grids of every size N in {8, 16, 32, 64}, mixed
    with a d = 1 window (which keeps the per-group stages), one-column passes
    included (row spreading, one-thread-per-point interpolation);
  * FP32, 32 right-hand sides in one pass (the benchmarked shape): the matvec
    equals the per-group stages, which the spectra call still runs (it keeps
    the forward spectrum), to FP32 rounding.
"""
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


@pytest.mark.parametrize("N3,N2,R,s", [(8, 64, 3, 4), (16, 32, 5, 5), (32, 16, 8, 5),
                                        (64, 16, 2, 5), (32, 64, 1, 4)])
def test_fp64_matches_oracle_nfft_fastsum(agp, N3, N2, R, s):
    rng = np.random.default_rng(N3 + 7 * N2 + R)
    n = 1500
    X = inputs.minmax_scale(rng.standard_normal((n, 6)))
    W = [[0, 1, 2], [3, 4], [5]]
    Ns = [N3, N2, 16]
    V = rng.standard_normal((n, R))
    plan = agp.Plan(torch.tensor(X, device=DEV), W, Ns, s, "matern12", 0.3, 0.8, 0.1)
    Vt = torch.tensor(V, device=DEV)
    got = plan.matvec(Vt).cpu().numpy()
    want = O.nfft_fastsum_matvec(X, W, "matern12", 0.3, 0.8, 0.1, V, Ns, s)
    assert rel(got, want) <= 1e-12
    # the ell-derivative multiplies by the derivative's coefficients
    gd = plan.deriv_matvec("ell", Vt).cpu().numpy()
    wd = O.truncated_deriv_matvec(X, W, "matern12", 0.3, 0.8, 0.1, V, Ns, "ell")
    assert rel(gd, wd) <= 1e-6
    plan.check()
    plan.close()


def test_fp32_benchmark_shape_matches_per_group_stages(agp):
    w = inputs.subset(inputs.nlml_grad(R=32), 20000)
    X = torch.tensor(w.X, dtype=torch.float32, device=DEV)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    plan = agp.Plan(X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    fused = plan.matvec(V)
    staged, _ = plan.spectra(V, out=True)
    plan.check()
    assert float((fused - staged).norm() / staged.norm()) <= 2e-6
    plan.close()
