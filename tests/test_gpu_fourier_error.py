"""The Fourier approximation error of Sec. 4 measured through the library: for
10^4 points r uniform in [-1/4, 1/4)^3, kappa_RF(r) = Re sum_{k in I_N} b_k
e^{2 pi i k.r} is evaluated by the library's NFFT from the library's own
coefficients b_k and compared with the exact kernel. The measured maximum
error must stay below the bounds of the Theorems of Sec. 4 for the
trivariate Matern(1/2) kernel and its ell-derivative (the paper states that
the bound holds for every ell it examined, and is tight when ell pi N > 1)."""
import math

import numpy as np
import pytest

import oracle as O

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


def bound_matern(ell, N):
    return 8.0 / (math.pi ** 2 * ell * (N - 2.0 * math.sqrt(3.0)))


def bound_matern_der(ell, N):
    m = N - 2.0 * math.sqrt(3.0)
    return 32.0 / (ell ** 4 * math.pi ** 4 * 3.0 * m ** 3) + 8.0 / (ell ** 2 * math.pi ** 2 * m)


@pytest.mark.parametrize("N", [16, 32, 64])
@pytest.mark.parametrize("ell", [0.05, 0.1, 0.3, 1.0])
def test_matern_fourier_error_within_theorem_bounds(agp, N, ell):
    rng = np.random.default_rng(N)
    R = rng.uniform(-0.25, 0.25, size=(10000, 3))
    plan = agp.Plan(torch.tensor(R, device=DEV), [[0, 1, 2]], N, 6, "matern12", ell, 1.0, 0.0)
    r = np.linalg.norm(R, axis=1)
    for der, exact, bound in ((False, O.kernel("matern12", r, ell), bound_matern(ell, N)),
                              (True, O.kernel_der_ell("matern12", r, ell),
                               bound_matern_der(ell, N))):
        b = plan.coeffs(0, der)
        fh = torch.tensor(b[None].astype(np.complex128), device=DEV)
        approx = plan.nfft_real(0, fh)[:, 0].cpu().numpy()
        err = float(np.max(np.abs(approx - exact)))
        assert err <= bound, (N, ell, der, err, bound)
