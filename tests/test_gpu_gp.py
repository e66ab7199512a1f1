"""GP training and prediction on top of the library (Sec. 5 settings): the
posterior mean against the oracle's dense solve on the Fourier-truncated
kernel, and Adam on the NLML estimate lowering the exact NLML."""
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
def gp():
    from paper_2504_00480_gb300 import agp as A
    from paper_2504_00480_gb300 import build
    from paper_2504_00480_gb300 import gp as G
    build.build()
    A.load_library()
    return G


def inv_softplus(v):
    return math.log(math.expm1(v))


def data(n, seed):
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((n, 4))
    y = np.sin(2.0 * raw[:, 0]) * np.cos(raw[:, 1]) + 0.5 * raw[:, 2] * raw[:, 3] \
        + 0.1 * rng.standard_normal(n)
    return inputs.minmax_scale(raw), y


def o2_dense(X, W, kind, ell, sf, se, N):
    n = X.shape[0]
    M = np.zeros((n, n))
    for a in range(0, n, 250):
        E = np.zeros((n, min(250, n - a)))
        E[np.arange(a, a + E.shape[1]), np.arange(E.shape[1])] = 1.0
        M[:, a:a + E.shape[1]] = O.truncated_matvec(X, W, kind, ell, sf, se, E, N)
    return 0.5 * (M + M.T)


def test_posterior_mean_matches_oracle(gp):
    X, y = data(1000, 3)
    Xtr, ytr, Xte = X[:800], y[:800], X[800:]
    W = [[0, 1], [2, 3]]
    th = (0.12, 0.9, 0.3)
    model = gp.AdditiveGP(Xtr, ytr, W, "gauss", 32, 5, dtype=torch.float64,
                          raw_init=[inv_softplus(v) for v in th])
    mean = model.predict(Xte, cg_iters=2000, rtol=1e-11)
    K = o2_dense(Xtr, W, "gauss", *th, 32)
    alpha = np.linalg.solve(K, ytr)
    V = np.concatenate([alpha, np.zeros(200)])[:, None]
    want = O.truncated_matvec(np.concatenate([Xtr, Xte]), W, "gauss", *th, V, 32,
                              rows=np.arange(800, 1000), add_noise=False)[:, 0]
    assert np.linalg.norm(mean - want) <= 1e-6 * np.linalg.norm(want)


@pytest.mark.parametrize("preconditioned", [True, False])
def test_adam_lowers_exact_nlml(gp, preconditioned):
    X, y = data(600, 5)
    W = [[0, 1], [2, 3]]
    # ell stays small enough for the truncated Gaussian to keep K_hat
    # positive definite (its most negative coefficient grows with ell)
    init = (0.15, 0.7, 0.7)
    model = gp.AdditiveGP(X, y, W, "gauss", 32, 5, dtype=torch.float32,
                          raw_init=[inv_softplus(v) for v in init])

    def exact(th):
        return O.nlml_exact(o2_dense(X, W, "gauss", *th, 32), y)

    before = exact(init)
    model.fit(iters=40, lr=0.03, n_probes=10, lanczos_steps=10, preconditioned=preconditioned)
    after = exact(model.hyper())
    assert after < before - 1e-3 * abs(before), (before, after, model.hyper())
