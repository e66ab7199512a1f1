"""GPU parity of batched independent problems (uneven n, per-problem
lengthscale): one launch per stage for all problems, also replayed from a
captured CUDA graph, against the oracle's truncated sum of every problem."""
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


@pytest.fixture(scope="module")
def problems(agp):
    # uneven-batch workload shape at oracle-sized n: 6 problems, n in [500, 3000]
    ws = inputs.uneven_batch(n_problems=6, n_lo=500, n_hi=3000, R=3)
    plans = [agp.Plan(torch.tensor(w.X, dtype=torch.float32, device=DEV), w.windows, w.N,
                      w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps) for w in ws]
    return ws, plans


@pytest.mark.parametrize("which", [None, "ell", "sigma_f", "sigma_eps"])
def test_batch_matches_oracle(agp, problems, which):
    ws, plans = problems
    batch = agp.Batch(plans)
    Vs = [torch.tensor(w.V, dtype=torch.float32, device=DEV) for w in ws]
    Outs = [torch.full_like(v, float("nan")) for v in Vs]
    batch.bind(Vs, Outs)
    batch.matvec(which)
    torch.cuda.synchronize()
    for w, out in zip(ws, Outs):
        if which is None:
            ref = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, w.V, w.N)
        else:
            ref = O.truncated_deriv_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                                           w.V, w.N, which)
        assert rel(out.cpu().numpy(), ref) <= 1e-4, w.name
    batch.close()


def test_batch_equals_single_plans_and_graph_replay(agp, problems):
    ws, plans = problems
    batch = agp.Batch(plans)
    Vs = [torch.tensor(w.V, dtype=torch.float32, device=DEV) for w in ws]
    Outs = [torch.zeros_like(v) for v in Vs]
    batch.bind(Vs, Outs)
    batch.matvec()                        # once outside capture
    torch.cuda.synchronize()
    singles = [p.matvec(v) for p, v in zip(plans, Vs)]
    for a, b in zip(Outs, singles):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6
    # capture the batch in a CUDA graph and replay it on new inputs
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.matvec()                    # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        batch.matvec()
    rng = np.random.default_rng(7)
    for _ in range(2):
        newV = [rng.standard_normal(v.shape) for v in Vs]
        for v, nv in zip(Vs, newV):
            v.copy_(torch.tensor(nv, dtype=torch.float32))
        g.replay()
        torch.cuda.synchronize()
        for w, out, nv in zip(ws, Outs, newV):
            ref = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, nv, w.N)
            assert rel(out.cpu().numpy(), ref) <= 1e-4
    batch.close()


def test_batch_rejects_mixed_cutoff(agp, problems):
    ws, plans = problems
    w = ws[0]
    other = agp.Plan(torch.tensor(w.X, dtype=torch.float32, device=DEV), w.windows, w.N, 5)
    with pytest.raises(agp.AgpError) as ei:
        agp.Batch([plans[0], other])
    assert ei.value.status == agp.AGP_EINVAL


def test_uneven_batch_full_size_sampled(agp):
    # The full uneven-batch workload: 64 problems, n log-uniform in
    # [1e4, 2e5] (~4e6 points), per-problem lengthscale, matvec and
    # ell-derivative matvec in one batched launch per stage, captured in a
    # CUDA graph. Checked on sampled rows of the three smallest problems and
    # the largest one against the oracle's truncated sum (all n points).
    ws = inputs.uneven_batch()
    assert len(ws) == 64 and sum(w.X.shape[0] for w in ws) > 3_000_000
    plans = [agp.Plan(torch.tensor(w.X, dtype=torch.float32, device=DEV), w.windows, w.N,
                      w.cutoff, w.kernel, w.ell, w.sigma_f, w.sigma_eps) for w in ws]
    Vs = [torch.tensor(w.V, dtype=torch.float32, device=DEV) for w in ws]
    Outs = [torch.zeros_like(v) for v in Vs]
    Ders = [torch.zeros_like(v) for v in Vs]
    b_mv, b_der = agp.Batch(plans), agp.Batch(plans)
    b_mv.bind(Vs, Outs)
    b_der.bind(Vs, Ders)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b_mv.matvec()
        b_der.matvec("ell")
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        b_mv.matvec()
        b_der.matvec("ell")
    for o in Outs + Ders:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    order = np.argsort([w.X.shape[0] for w in ws])
    rng = np.random.default_rng(11)
    for q in list(order[:3]) + [order[-1]]:
        w = ws[q]
        rows = np.sort(rng.choice(w.X.shape[0], 16, replace=False))
        ref = O.truncated_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps, w.V,
                                 w.N, rows=rows)
        assert rel(Outs[q].cpu().numpy()[rows], ref) <= 1e-4, w.name
        dref = O.truncated_deriv_matvec(w.X, w.windows, w.kernel, w.ell, w.sigma_f, w.sigma_eps,
                                        w.V, w.N, "ell", rows=rows)
        assert rel(Ders[q].cpu().numpy()[rows], dref) <= 1e-4, w.name
    b_mv.close()
    b_der.close()
