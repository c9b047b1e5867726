"""The allocation-free forward projection (wmg_project_noalloc): for callers
that cannot allocate device memory while they run (memory reserved up front
so nothing can fail or stall mid-scan, or a framework allocator that already
holds all free memory). It must give the same sinogram as the plan-based
wmg_project bit for bit (same angle tables, same kernel), call after call,
although every call reuses the same fixed scratch arrays; the sinogram
matches the FP64 oracle's W x to FP32 rounding; and after the first call on
the device, which loads the arrays, calls take no device memory. Collected
last so that a run that stops at the first failure has already run every
other test."""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu


def project_noalloc(n, m, D, x, b):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = wmg.lib().wmg_project_noalloc(n, m, D, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                       stream)
    assert rc == 0, wmg.last_error()
    return b


@pytest.mark.parametrize("n,m,D", [(256, 180, 363), (64, 90, 91), (33, 20, 48)])
def test_noalloc_matches_plan_projection_twice(n, m, D):
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32)
    op = oracle.Op(n, m, D)
    rng = np.random.default_rng(n + m)
    b = torch.empty(m * D, dtype=torch.float32, device="cuda")
    for call in range(2):                      # two calls in a row share the scratch
        xh = rng.random(n * n).astype(np.float32)
        x = torch.tensor(xh, device="cuda")
        ref = plan.project(x)
        got = project_noalloc(n, m, D, x, b)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        assert np.array_equal(got, ref), call
        exact = op.project(xh.astype(np.float64))
        assert np.abs(got - exact).max() <= 1e-6 * np.abs(exact).max(), call
    plan.close()


def test_noalloc_takes_no_device_memory_after_its_first_call():
    n, m, D = 128, 60, 182
    x = torch.rand(n * n, dtype=torch.float32, device="cuda")
    b1 = torch.empty(m * D, dtype=torch.float32, device="cuda")
    b2 = torch.empty_like(b1)
    project_noalloc(n, m, D, x, b1)            # the first call on this device loads the arrays
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        project_noalloc(n, m, D, x, b2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(b1, b2)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = wmg.lib().wmg_project_noalloc(2048, 10, 10, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), None)
    assert rc == -1 and "1024" in wmg.last_error()
