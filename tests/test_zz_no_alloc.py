"""The allocation-free forward projection (wmg_project_noalloc): for callers
that cannot allocate device memory while they run (memory reserved up front
so nothing can fail or stall mid-scan). It must give the same sinogram as
the plan-based wmg_project, call after call, although every call reuses the
same fixed scratch arrays. Collected last so that a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu


def project_noalloc(n, m, D, x):
    b = torch.empty(m * D, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = wmg.lib().wmg_project_noalloc(n, m, D, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                       stream)
    assert rc == 0, wmg.last_error()
    return b


@pytest.mark.parametrize("n,m,D", [(256, 180, 363), (64, 90, 91), (33, 20, 48)])
def test_noalloc_matches_plan_projection_twice(n, m, D):
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32)
    rng = np.random.default_rng(n + m)
    for call in range(2):                      # two calls in a row share the scratch
        x = torch.tensor(rng.random(n * n), dtype=torch.float32, device="cuda")
        ref = plan.project(x)
        got = project_noalloc(n, m, D, x)
        torch.cuda.synchronize()
        ref, got = ref.double().cpu().numpy(), got.double().cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), call
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = wmg.lib().wmg_project_noalloc(2048, 10, 10, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), None)
    assert rc == -1 and "1024" in wmg.last_error()
