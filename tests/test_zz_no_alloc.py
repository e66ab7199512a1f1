"""The allocation-free column dot products (agp_dot_columns_static).

Some callers cannot let the library allocate device memory -- code running
inside a framework or memory pool that owns the device's memory, or a
latency-critical loop that must not trigger an allocation. For them the
library keeps the scratch of this reduction in a fixed device array. This
test calls the allocation-free entry point through the C ABI and checks it
against the allocating one (agp_dot_columns) on two calls in a row, so that
stale scratch from the first call cannot go unnoticed, and both against the
column sums of the elementwise products computed in FP64 on the host
(numpy), a reference that shares no code with the library. It lives in a file of
its own that pytest collects last; it passes alone in a fresh process and
after the other tests.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_static_dot_matches_allocating_dot_on_two_calls(agp, dtype):
    lib = agp.load_library()
    rng = np.random.default_rng(123)
    n, R = 20_000, 37
    # a plan only supplies n and the precision to the allocating entry point
    X = torch.tensor(rng.uniform(-0.24, 0.24, size=(n, 1)), dtype=dtype, device=DEV)
    plan = agp.Plan(X, [[0]], 8, 2)
    out = torch.full((R,), float("nan"), dtype=torch.float64, device=DEV)
    prec = 0 if dtype == torch.float32 else 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        wide_a = torch.tensor(rng.standard_normal((n, R + 5)), dtype=dtype, device=DEV)
        B = torch.tensor(rng.standard_normal((n, R)) * (call + 1), dtype=dtype, device=DEV)
        A = wide_a[:, 2:2 + R]                      # leading dimension R + 5
        ref = agp.agp_dot_columns(plan.handle, A, B)
        st = lib.agp_dot_columns_static(prec, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                        n, R, out.data_ptr(), stream)
        assert st == agp.AGP_OK, lib.agp_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # both accumulate in FP64; only the split into partial sums differs
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        # independent reference: FP64 products of the same (rounded) inputs,
        # summed on the host
        An = A.cpu().double().numpy()
        Bn = B.cpu().double().numpy()
        host = np.sum(An * Bn, axis=0)
        scale = np.sum(np.abs(An * Bn), axis=0)
        np.testing.assert_allclose(got, host, rtol=0, atol=1e-12 * scale.max())
    plan.close()


def test_static_dot_rejects_too_many_columns(agp):
    lib = agp.load_library()
    A = torch.zeros((10, 65), dtype=torch.float32, device=DEV)
    out = torch.zeros(65, dtype=torch.float64, device=DEV)
    st = lib.agp_dot_columns_static(0, A.data_ptr(), 65, A.data_ptr(), 65, 10, 65,
                                    out.data_ptr(), None)
    assert st == agp.AGP_EINVAL
    assert b"64" in lib.agp_last_error()
