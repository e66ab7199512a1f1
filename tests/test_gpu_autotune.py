"""The work-item size (points per CTA of spreading/interpolation) is a layout
choice with no effect on the operator: results must not depend on it, and the
autotuner must keep one of its candidates."""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 2e-6), (torch.float64, 1e-13)])
def test_item_points_do_not_change_results(agp, dtype, tol):
    w = inputs.subset(inputs.nlml_grad(n=60000, R=17), 60000)
    plan = agp.Plan(torch.tensor(w.X, dtype=dtype, device=DEV), w.windows, w.N, w.cutoff,
                    w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    V = torch.tensor(w.V, dtype=dtype, device=DEV)
    ref = plan.matvec(V).cpu().numpy()
    dref = plan.deriv_matvec("ell", V).cpu().numpy()
    # work items of window 0: ceil(count / size) per occupied grid cell
    _, counts = np.unique(O.bins(w.X[:, w.windows[0]], 2 * w.N[0]), axis=0, return_counts=True)
    assert plan.query(0)["n_items"] == int(np.sum(-(-counts // 256)))
    for pts in (4, 100, 4096):
        plan.set_item_points(max(pts, 16))
        assert plan.query(0)["n_items"] == int(np.sum(-(-counts // max(pts, 16))))
        assert plan.matvec(V).cpu().numpy() == pytest.approx(ref, rel=0, abs=tol * np.abs(ref).max())
        assert rel(plan.deriv_matvec("ell", V).cpu().numpy(), dref) <= tol
    plan.set_item_points(16)
    want = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                              w.V[:, :1], w.N)
    got = plan.matvec(V[:, :1].contiguous()).cpu().numpy()
    assert rel(got, want) <= (1e-4 if dtype == torch.float32 else 1e-9)


def test_autotune_keeps_a_candidate(agp):
    agp.load_library().agp_autotune_clear_cache()
    w = inputs.subset(inputs.nlml_grad(n=40000, R=8), 40000)
    plan = agp.Plan(torch.tensor(w.X, dtype=torch.float32, device=DEV), w.windows, w.N, w.cutoff,
                    w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    ref = plan.matvec(V).cpu().numpy()
    pts, ms = plan.autotune(R=8, reps=2)
    assert pts in (64, 128, 256, 512, 1024) and ms > 0
    assert plan.tensor_cores() in (0, 1, 2, 3)
    assert rel(plan.matvec(V).cpu().numpy(), ref) <= 2e-6
    # a batch created after the autotuner uses the new items
    b = agp.Batch([plan])
    out = torch.empty_like(V)
    b.bind([V], [out])
    b.matvec()
    assert rel(out.cpu().numpy(), ref) <= 2e-6


def test_item_points_rejected(agp):
    w = inputs.subset(inputs.nlml_grad(n=3000, R=1), 3000)
    plan = agp.Plan(torch.tensor(w.X, dtype=torch.float32, device=DEV), w.windows, w.N, w.cutoff,
                    w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    for pts in (8, 5000):
        with pytest.raises(agp.AgpError) as ei:
            plan.set_item_points(pts)
        assert ei.value.status == agp.AGP_EINVAL


def test_autotune_family_and_cache(agp):
    """With 32 right-hand sides the tensor-core families compete with the FMA
    pipes; the choice is one of them, leaves the operator unchanged, and a
    second plan of the same shape takes the cached choice."""
    agp.load_library().agp_autotune_clear_cache()
    w = inputs.subset(inputs.nlml_grad(n=50000, R=32), 50000)
    mk = lambda: agp.Plan(torch.tensor(w.X, dtype=torch.float32, device=DEV), w.windows, w.N,
                          w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps)
    plan = mk()
    V = torch.tensor(w.V, dtype=torch.float32, device=DEV)
    plan.set_tensor_cores(0)
    ref = plan.matvec(V).cpu().numpy()
    pts, ms = plan.autotune(R=32, reps=2)
    mode = plan.tensor_cores()
    assert mode in (0, 1, 2, 3) and pts in (64, 128, 256, 512, 1024)
    assert rel(plan.matvec(V).cpu().numpy(), ref) <= 1e-5
    other = mk()
    pts2, ms2 = other.autotune(R=32, reps=2)
    assert (pts2, ms2, other.tensor_cores()) == (pts, ms, mode)
    plan.close()
    other.close()
