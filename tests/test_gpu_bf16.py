"""BF16 operator storage (WMG_PREC_F32_BF16STORE): inside the Arnoldi steps
of preconditioned GMRES the operator's stored inputs are bfloat16 (FP32
arithmetic and accumulation, FP64 Krylov vectors and Gram-Schmidt); every
restart recomputes the true residual with the FP32 operator (residual
replacement). The rounded inputs perturb the Arnoldi relation by about 2^-9,
so the iterates follow another Krylov path than the FP32 plan's: the test is
that the path still converges to the requested 1e-4, checked by the FP64
oracle's own normal-equation residual of the returned image, within twice
the FP32 plan's iterations; and that the other solvers and the operator
calls of such a plan are the FP32 plan's bit for bit."""
import numpy as np
import pytest

import oracle
import oracle_jobs as J
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

COUNT = 8


@pytest.fixture(scope="module")
def mid():
    probs = S.workload_mid(COUNT).problems
    op = oracle.Op(probs[0].n, probs[0].m, probs[0].D)
    bs = np.stack([J.noisy_sinogram(p, op) for p in probs])
    return probs, op, bs


def plan(P, precision):
    return wmg.Plan(P.n, P.m, P.D, levels=5, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=precision)


def test_bf16_storage_gmres_reaches_the_tolerance(mid):
    probs, op, bs = mid
    b = torch.tensor(bs.reshape(-1), dtype=torch.float32, device="cuda")
    p32, p16 = plan(probs[0], wmg.PREC_F32), plan(probs[0], wmg.PREC_F32_BF16STORE)
    _, info32, _, _ = p32.solve(b, wmg.SOLVER_GMRES, True, max_iter=200, rtol=1e-4, restart=20)
    x16, info16, _, rc = p16.solve(b, wmg.SOLVER_GMRES, True, max_iter=200, rtol=1e-4, restart=20)
    torch.cuda.synchronize()
    x16 = x16.double().cpu().numpy().reshape(COUNT, -1)
    assert rc == 0
    for i in range(COUNT):
        assert info16[i][1] == 0 and info16[i][2] < 1e-4
        assert info16[i][0] <= 2 * info32[i][0]
        # the FP64 oracle's residual of the returned image: FP32 rounding of
        # the output image and of the sinogram on top of the 1e-4 the solve
        # confirmed with its FP32 operator
        assert op.ne_residual(bs[i], x16[i]) < 1.1e-4
    p32.close()
    p16.close()


def test_bf16_plan_runs_the_other_solvers_as_fp32(mid):
    probs, op, bs = mid
    b = torch.tensor(bs[:2].reshape(-1), dtype=torch.float32, device="cuda")
    outs = []
    for prec in (wmg.PREC_F32, wmg.PREC_F32_BF16STORE):
        pl = plan(probs[0], prec)
        pa = wmg.Plan(probs[0].n, probs[0].m, probs[0].D, levels=5, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE,
                      precision=prec)
        xc, _, _, _ = pa.solve(b, wmg.SOLVER_CGLS, True, max_iter=6, rtol=0.0)
        xg, _, _, _ = pl.solve(b, wmg.SOLVER_GMRES, False, max_iter=6, rtol=0.0)
        q = pl.project(xc)
        y = pl.backproject(b)
        torch.cuda.synchronize()
        outs.append([t.clone() for t in (xc, xg, q, y)])
        pl.close()
        pa.close()
    for a_, b_ in zip(*outs):
        assert torch.equal(a_, b_)


def test_bf16_storage_is_refused_by_batches():
    with pytest.raises(wmg.WmgError) as e:
        wmg.Batch([dict(n=64, m=30, D=91, levels=3)], nu1=0, nu2=0, precision=wmg.PREC_F32_BF16STORE)
    assert e.value.code == wmg.WMG_ERR_INVALID_ARG
