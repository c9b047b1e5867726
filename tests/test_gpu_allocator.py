"""The caller's workspace allocator (wmg_set_allocator) on the GPU: with
torch's caching allocator installed, a plan's workspace is torch memory
(counted by torch.cuda.memory_allocated while the plan lives, all of it
returned when the plan is destroyed) and its results are bitwise those of
a plan on cudaMalloc; an allocator that refuses makes plan creation fail
with WMG_ERR_OOM."""
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

P = S.workload_small().problems[0]


def gmres(prec):
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    b = torch.tensor(oracle.Op(P.n, P.m, P.D).project(P.image()), dtype=dt, device="cuda")
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=prec)
    x, info, hist, _ = plan.solve(b, wmg.SOLVER_GMRES, True, 10, 0.0, 5, history=True)
    torch.cuda.synchronize()
    return plan, x, info, hist[0]


@pytest.mark.parametrize("prec", [wmg.PREC_F64, wmg.PREC_F32])
def test_workspace_in_torch_memory(prec):
    plan, x_ref, info_ref, hist_ref = gmres(prec)
    plan.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    wmg.use_torch_allocator(True)
    try:
        plan, x, info, hist = gmres(prec)
        held = torch.cuda.memory_allocated() - before - x.numel() * x.element_size()
        # at least the FP64 Arnoldi basis of GMRES(5): 6 vectors of N doubles
        assert held >= 6 * P.n * P.n * 8
        assert torch.equal(x, x_ref) and info == info_ref and (hist == hist_ref).all()
        plan.close()
        del x
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        wmg.use_torch_allocator(False)


def test_refusing_allocator_is_out_of_memory():
    alloc = wmg._ALLOC_FN(lambda nbytes, stream, ctx: None)
    free = wmg._FREE_FN(lambda ptr, nbytes, stream, ctx: None)
    wmg.wmg_set_allocator(alloc, free)
    try:
        with pytest.raises(wmg.WmgError) as e:
            wmg.Plan(P.n, P.m, P.D, levels=3)
        assert e.value.code == wmg.WMG_ERR_OOM
    finally:
        wmg.wmg_set_allocator(None, None)
    # cudaMalloc again
    wmg.Plan(P.n, P.m, P.D, levels=3).close()
