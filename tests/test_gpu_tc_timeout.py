"""Bounded waits of the tensor-core kernels: with a wait limit of one poll
the mbarrier waits for MMAs that were just issued give up, every CTA agrees
on it, drains its MMAs, skips its epilogue and releases its tensor memory.
The library then reports AGP_TIMEOUT -- through agp_plan_check after an
asynchronous matvec and directly from the entry points that synchronise --
and, with the default limit restored, the same plan computes the right
result again (the device stayed usable)."""
import numpy as np
import pytest

import oracle as O
from paper_2504_00480_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]
DEV = "cuda:0"
AGP_TIMEOUT = 6


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


def make(agp, n=6000, R=32, seed=11):
    rng = np.random.default_rng(seed)
    X = inputs.to_precision(inputs.minmax_scale(rng.standard_normal((n, 6))),
                            np.float32).astype(np.float64)
    W = [[0, 1, 2], [3, 4, 5]]
    V = rng.standard_normal((n, R))
    plan = agp.Plan(torch.tensor(X, dtype=torch.float32, device=DEV), W, 32, 5, "gauss",
                    0.2, 1.0, 0.3)
    plan.set_tensor_cores(True)
    return plan, X, W, V, torch.tensor(V, dtype=torch.float32, device=DEV)


def test_expired_wait_is_reported_and_the_plan_recovers(agp):
    plan, X, W, V, Vt = make(agp)
    plan.set_wait_limit(1)
    plan.matvec(Vt)
    torch.cuda.synchronize()
    with pytest.raises(agp.AgpError) as e:
        plan.check()
    assert e.value.status == AGP_TIMEOUT
    plan.check()                      # the flag was cleared by the report
    plan.set_wait_limit(0)            # default limit
    got = plan.matvec(Vt).cpu().numpy()
    plan.check()
    want = O.truncated_matvec(X, W, "gauss", 0.2, 1.0, 0.3, V, 32)
    assert rel(got, want) <= 1e-4
    plan.close()


def test_synchronising_entry_points_return_timeout(agp):
    plan, X, W, V, Vt = make(agp, n=4000, R=17, seed=12)
    B = Vt[:, :17].contiguous()
    Xs = torch.zeros_like(B)
    plan.set_wait_limit(1)
    with pytest.raises(agp.AgpError) as e:
        agp.agp_pcg_solve(plan.handle, B, Xs, rtol=1e-6, maxit=3)
    assert e.value.status == AGP_TIMEOUT
    with pytest.raises(agp.AgpError) as e:
        plan.nlml_grad(B[:, 0].contiguous(), B[:, 1:17], lanczos_steps=3)
    assert e.value.status == AGP_TIMEOUT
    plan.set_wait_limit(0)
    it, rr = agp.agp_pcg_solve(plan.handle, B, Xs, rtol=1e-6, maxit=3,
                               raise_not_converged=False)
    assert (it == 3).all() and np.isfinite(rr).all()
    plan.check()
    plan.close()


def test_wait_limit_rejects_negative(agp):
    plan, *_ = make(agp, n=500, R=1, seed=13)
    with pytest.raises(agp.AgpError):
        plan.set_wait_limit(-1)
    plan.close()
