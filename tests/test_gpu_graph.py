"""A plan's matvec captured in a CUDA graph and replayed: the benchmarked
window shapes (d = 3, 3, 2), whose d = 2 window runs on the plan's second
stream next to the d = 3 launches (forked from and joined to the capturing
stream by events), FP32, 32 right-hand sides. The replay must equal the
eager call on the same inputs and follow new inputs copied into the captured
buffer."""
import numpy as np
import pytest

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


def test_plan_matvec_replays_from_a_cuda_graph(agp):
    w = inputs.subset(inputs.nlml_grad(R=32), 50000)
    X = torch.tensor(w.X, dtype=torch.float32, device=DEV)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    plan = agp.Plan(X, w.windows, w.N, w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    assert plan.kernel_families(32) == (3, 3)
    Out = torch.empty_like(V)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        agp.agp_matvec(plan.handle, V, Out, True)      # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        agp.agp_matvec(plan.handle, V, Out, True)
    rng = np.random.default_rng(11)
    for _ in range(2):
        V.copy_(torch.tensor(rng.standard_normal(tuple(V.shape)), dtype=torch.float32))
        g.replay()
        torch.cuda.synchronize()
        ref = plan.matvec(V)
        assert float((Out - ref).norm() / ref.norm()) <= 2e-6
    plan.check()
    plan.close()
