"""WMG-BiCGStab (the solver of the paper's experiments, Section 4) on the GPU
against the oracle's BiCGStab: iterates after a fixed count (FP64 1e-10
preconditioned; a few iterations unpreconditioned, where rounding grows),
convergence to a tolerance, FP32 mixed path within 1e-4, and a problem alone
equal to the same problem in a batch."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

W = S.workload_small()
P = W.problems[0]


def data(prob=P, noise=0.0):
    op = oracle.Op(prob.n, prob.m, prob.D)
    b = op.project(prob.image())
    if noise:
        b = b + noise * np.abs(b).max() * prob.noise_unit()
    return op, b


@pytest.mark.parametrize("cycle,hd", [(oracle.CYCLE_HYBRID, 1), (oracle.CYCLE_ADDITIVE, 0)])
def test_preconditioned_matches_oracle_f64(cycle, hd):
    op, b = data()
    lam = 0.0
    M = oracle.Wmg(op, 3, 1, 1, 1.0, lam, cycle, hd)
    x_ref, k, hist_ref, st = oracle.bicgstab(op, b, 12, 0.0, lam, M)
    assert k == 12
    # the oracle's own rounding sensitivity: the same run with every sum
    # reversed (BiCGStab amplifies rounding more than GMRES, more so with the
    # weaker additive cycle); the GPU must agree to 1e-10 or within 20x that
    oracle.set_reverse_summation(True)
    try:
        x_rev, _, _, _ = oracle.bicgstab(op, b, 12, 0.0, lam, M)
    finally:
        oracle.set_reverse_summation(False)
    floor = np.linalg.norm(x_rev - x_ref) / np.linalg.norm(x_ref)
    tol = max(1e-10, 20 * floor)
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=1, nu2=1, hybrid_depth=hd, cycle=cycle, precision=wmg.PREC_F64)
    x, info, hists, rc = plan.solve(torch.tensor(b, device="cuda"), wmg.SOLVER_BICGSTAB, True, 12, 0.0,
                                    history=True)
    assert info[0][0] == 12
    x = x.cpu().numpy()
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < tol, (floor, tol)
    np.testing.assert_allclose(hists[0], hist_ref, rtol=max(1e-8, 100 * floor), atol=1e-14)
    # the first iterations, before rounding grows, agree tightly
    x3, _, _, _ = plan.solve(torch.tensor(b, device="cuda"), wmg.SOLVER_BICGSTAB, True, 3, 0.0)
    x3_ref, _, _, _ = oracle.bicgstab(op, b, 3, 0.0, lam, M)
    assert np.linalg.norm(x3.cpu().numpy() - x3_ref) / np.linalg.norm(x3_ref) < 1e-12


def test_unpreconditioned_first_iterations_f64():
    op, b = data()
    x_ref, k, hist_ref, st = oracle.bicgstab(op, b, 4, 0.0, 0.0, None)
    plan = wmg.Plan(P.n, P.m, P.D, levels=3, precision=wmg.PREC_F64)
    x, info, hists, rc = plan.solve(torch.tensor(b, device="cuda"), wmg.SOLVER_BICGSTAB, False, 4, 0.0,
                                    history=True)
    assert np.linalg.norm(x.cpu().numpy() - x_ref) / np.linalg.norm(x_ref) < 1e-10
    np.testing.assert_allclose(hists[0], hist_ref, rtol=1e-9, atol=1e-14)


def test_converges_to_tolerance_and_f32_path():
    op, b = data(noise=0.01)
    lam = 1e-3 * P.m / P.n
    M = oracle.Wmg(op, 3, 0, 0, 1.0, lam, oracle.CYCLE_HYBRID, 1)
    x_ref, k, hist_ref, st = oracle.bicgstab(op, b, 200, 1e-6, lam, M)
    assert st == 0
    # FP64: to the tolerance, the oracle's iteration count and iterate;
    # FP32 mixed path: the same iteration count, within 1e-4 of the oracle
    for prec, tol, rtol in ((wmg.PREC_F64, 1e-8, 1e-6), (wmg.PREC_F32, 1e-4, 0.0)):
        dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
        plan = wmg.Plan(P.n, P.m, P.D, levels=3, nu1=0, nu2=0, lam=lam, hybrid_depth=1,
                        cycle=wmg.CYCLE_HYBRID, precision=prec)
        x, info, _, rc = plan.solve(torch.tensor(b, dtype=dt, device="cuda"), wmg.SOLVER_BICGSTAB, True,
                                    200 if rtol else k, rtol)
        assert info[0][0] == k
        if rtol:
            assert info[0][1] == wmg.WMG_OK and info[0][2] < rtol
        xn = x.double().cpu().numpy()
        assert np.linalg.norm(xn - x_ref) / np.linalg.norm(x_ref) < tol


def test_batch_equals_alone():
    n, m, D = 64, 36, 91
    op = oracle.Op(n, m, D)
    bs = np.stack([op.project(S.phantom(n, 6, S.seed_for(8, i))) for i in range(10)])
    plan = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
    b = torch.tensor(bs.reshape(-1), dtype=torch.float32, device="cuda")
    x_all, info_all, _, _ = plan.solve(b, wmg.SOLVER_BICGSTAB, True, 30, 1e-5)
    single = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                      precision=wmg.PREC_F32)
    for i in range(10):
        x1, info1, _, _ = single.solve(b[i * m * D:(i + 1) * m * D].contiguous(), wmg.SOLVER_BICGSTAB, True, 30,
                                       1e-5)
        torch.cuda.synchronize()
        assert info1[0][:2] == info_all[i][:2]
        assert torch.equal(x1, x_all[i * n * n:(i + 1) * n * n]), i
